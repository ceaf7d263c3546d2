"""GPU parity: the sm_103a path through the C ABI against the FP64 oracle, element by element.

Bar (integers bit-exact; FP64 tallies within 1e-12 relative per cell; FP32 within 1e-4 relative on
cells above 1e-3 of the peak, with the FP32 error reported for every tally):
  * point sets (Sobol + digital shift, counter PRNG, PRNG fallback past the table) bit-exact
  * MC leg: per-history (final cell, fate, scatter count, segments) and all counters bit-exact,
    pre/post tallies and hand-off moments within the tolerance, balance
  * collided S_N-DG solve, remap (with the comb), and whole multi-step runs
Sizes span several S_N tiles and a ragged tail; edge cases: 1x1 mesh, one history, empty bank,
N_s = 0, killing, no source.
"""
import math

import numpy as np
import pytest

from paper_2511_16821_gb300 import workloads as W

pytestmark = pytest.mark.gpu

from parity_checks import (FP32_RTOL, FP32_RTOL_THICK, FP64_RTOL, check_counts, check_fp64_libm,  # noqa: E402
                           check_fp64_tallies, fp32_check, rel_err)


@pytest.fixture(scope="module")
def H():
    import torch
    from paper_2511_16821_gb300 import hyb
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hyb.lib()
    return hyb


def n_hist_total(spec, bank):
    nb = 0 if bank is None else int(bank["n"])
    return nb + (spec.n_hist if spec.Q is not None and np.sum(spec.Q) > 0 else 0)


def gpu_leg(H, spec, bank, step=0):
    import torch
    P = H.Problem(spec.with_(ic=None))
    P.set_bank(bank if bank is not None else {"cell": np.zeros(0, np.int32), **{k: np.zeros(0) for k in ("fx", "fy", "ox", "oy", "w")}, "n": 0})
    P.set_step(step)
    N = n_hist_total(spec, bank)
    tr = torch.full((max(N, 1), 4), -7, dtype=torch.int32, device="cuda")
    st = P.mc_leg(trace=tr)
    out = dict(pre=P.tally("pre_raw"), post=P.tally("post_raw"), mom=P.tally("handoff"), stats=st,
               hist=tr.cpu().numpy()[:N], P=P)
    return out


# ------------------------------------------------------------------------------------------------
# point sets
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("sampler", [0, 1, 2])
@pytest.mark.parametrize("i0,n,nd", [(0, 4097, 29), (123456, 3000, 70), (2 ** 31 - 5, 10, 8),
                                     (2 ** 32 - 3000, 3000, 65)])
def test_points_bitexact(H, orc, sampler, i0, n, nd):
    g = H.points(99, 7, 3, sampler, i0, n, nd).cpu().numpy().view(np.uint32)
    o = orc.points(99, 7, 3, sampler, i0, n, nd)
    assert np.array_equal(g, o)


# ------------------------------------------------------------------------------------------------
# integer 2-D CDF (birth and remap sampling map)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny", [(1, 1), (37, 5), (112, 112), (300, 2)])
def test_cdf_bitexact(H, orc, nx, ny):
    import torch
    rng = np.random.default_rng(nx * 1000 + ny)
    w = rng.uniform(-1, 1, nx * ny) ** 3
    w[rng.integers(0, nx * ny, max(1, nx * ny // 7))] = 0.0
    q, rp, cp, wq = H.build_cdf(torch.tensor(w, device="cuda"), nx, ny)
    oq, orp, ocp = orc.build_cdf(nx, ny, w)
    assert np.array_equal(q.cpu().numpy(), oq)
    assert np.array_equal(rp.cpu().numpy(), orp)
    assert np.array_equal(cp.cpu().numpy(), ocp)
    assert wq[1].item() == np.max(np.abs(w))
    assert math.isclose(wq[0].item(), float(np.sum(np.abs(w))), rel_tol=1e-13)


# ------------------------------------------------------------------------------------------------
# MC leg, FP64
# ------------------------------------------------------------------------------------------------
def leg_cases():
    cb = W.checkerboard(n_s=2, n_hist=20_000, cells_per_block=5)   # 35x35: ragged vs 32-tiles
    rng = np.random.default_rng(0)
    het = W.ProblemSpec(nx=37, ny=23, lx=3.7, ly=2.0, sigma_a=rng.uniform(0, 2, 37 * 23),
                        sigma_s=rng.uniform(0, 4, 37 * 23), Q=rng.uniform(0, 1, 37 * 23) ** 2, dt=0.3,
                        n_s=3, n_hist=30_000, seed=5, w_min=0.05)
    return [
        ("pulse", W.pulse(n_hist=10_000), "ic", 0),
        ("cb_ns0", cb.with_(n_s=0), 5000, 3),
        ("cb_ns1", cb.with_(n_s=1), 5000, 1),
        ("cb_ns2", cb, 5000, 2),
        ("cb_ns4_prng", cb.with_(n_s=4, sampler=W.PRNG), 5000, 4),
        ("cb_ns3_halton", cb.with_(n_s=3, sampler=W.HALTON), 5000, 5),
        ("cb_ns_cell", cb.with_(n_s=3, n_s_cell=np.random.default_rng(4).integers(0, 4, cb.ncells).astype(np.int32)),
         5000, 7),
        ("het_kill", het, 4000, 6),
        ("one_cell", W.homogeneous(n=1, L=0.5, sigma_a=0.3, sigma_s=2.0, Q=1.0, n_hist=1, dt=1.0, n_s=2), 1, 0),
        ("no_source_empty", W.homogeneous(n=3, Q=None, n_hist=5), 0, 0),
        ("n_s_20", W.homogeneous(n=6, L=1.0, sigma_a=0.1, sigma_s=30.0, Q=1.0, n_hist=3000, dt=0.5, n_s=20), 500, 1),
    ]


def gpu_leg_without(H, spec, bank, step, skip_idx):
    """The leg with the histories at global indices skip_idx left out: range legs over the gaps,
    their exchange blocks summed and finished (raw tallies as gpu_leg)."""
    P = H.Problem(spec.with_(ic=None))
    P.set_bank(bank if bank is not None else {"cell": np.zeros(0, np.int32), **{k: np.zeros(0) for k in ("fx", "fy", "ox", "oy", "w")}, "n": 0})
    P.set_step(step)
    total = P.exchange_block()
    lo = 0
    for h in sorted(int(x) for x in skip_idx) + [1 << 62]:
        if h > lo:
            blk = P.exchange_block()
            P.mc_leg_range(lo, h, blk)
            total += blk
        lo = h + 1
    st = P.mc_leg_reduce_finish(total)
    out = dict(pre=P.tally("pre_raw"), post=P.tally("post_raw"), mom=P.tally("handoff"), stats=st)
    P.close()
    return out


def fp32_without(H, orc, spec32, bank, step, run_oracle):
    """Regrade of an FP32 leg with some histories taken out of both sides."""
    def f(idx):
        n = int(orc.n_histories(spec32, bank))
        skip = np.zeros(n, np.uint8)
        skip[idx] = 1
        return gpu_leg_without(H, spec32, bank, step, idx), run_oracle(skip)
    return f


def bank_for(orc, spec, nb):
    if nb == "ic":
        return orc.init_bank(spec, spec.ic)
    if nb == 0:
        return None
    return W.random_bank(spec, nb, seed=nb + 1)


@pytest.mark.parametrize("case", leg_cases(), ids=lambda c: c[0])
def test_mc_leg_fp64_parity(H, orc, case):
    """FP64 path against the oracle evaluating the direction and optical-depth maps with the
    explicit series (the FP64 path's own recipe): every record and counter bit-exact, tallies to
    1e-12; and against the oracle on the host libm: records differ only at near ties (reported
    with their margins), tallies to 1e-12 beside the flipped histories."""
    name, spec, nb, step = case
    bank = bank_for(orc, spec, nb)
    g = gpu_leg(H, spec, bank, step)
    o = orc.mc_leg(spec, step, bank, want_hist=True, elem=orc.SERIES)
    assert o["rc"] in (0, 3)
    if g["hist"].size:
        mism = np.nonzero(np.any(g["hist"] != o["hist"], axis=1))[0]
        assert mism.size == 0, f"{mism.size} history records differ, first {mism[:5]}: " \
                               f"{g['hist'][mism[:3]]} vs {o['hist'][mism[:3]]}"
    check_counts(g["stats"], o["stats"])
    check_fp64_tallies(g, o)
    ol = orc.mc_leg(spec, step, bank, want_hist=True, want_margin=True, elem=orc.LIBM)
    check_fp64_libm(g, ol, spec, bank, name)


def test_initial_bank_parity(H, orc):
    spec = W.pulse(n_hist=4096)
    P = H.Problem(spec)
    g = P.bank()
    o = orc.init_bank(spec, spec.ic, elem=orc.SERIES)
    assert g["n"] == o["n"] == 4096
    assert np.array_equal(g["cell"], o["cell"])
    # the direction map follows the series recipe on both sides, so the bank is identical
    for k in ("fx", "fy", "ox", "oy", "w"):
        assert np.array_equal(g[k], o[k]), k
    # against the libm maps: cells and positions are integer-CDF picks (identical), directions
    # agree to the maps' rounding
    ol = orc.init_bank(spec, spec.ic, elem=orc.LIBM)
    assert np.array_equal(g["cell"], ol["cell"])
    for k in ("fx", "fy", "w"):
        assert np.array_equal(g[k], ol[k]), k
    for k in ("ox", "oy"):
        assert np.max(np.abs(g[k] - ol[k])) < 2e-15, k


# ------------------------------------------------------------------------------------------------
# MC leg, FP32 tracking (cell-local coordinates, int64 fixed-point tallies)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("case", [c for c in leg_cases() if c[0] in ("pulse", "cb_ns0", "cb_ns2", "het_kill",
                                                                     "cb_ns3_halton", "cb_ns_cell")],
                         ids=lambda c: c[0])
def test_mc_leg_fp32_tolerance(H, orc, case):
    """FP32 tracking vs the FP64 oracle (libm maps): 1e-4 relative on every resolved cell above
    1e-3 of the peak, the unrestricted maximum bounded, flips reported with their margins."""
    name, spec, nb, step = case
    bank = bank_for(orc, spec, nb)
    o = orc.mc_leg(spec, step, bank, want_hist=True, want_margin=True)
    s32 = spec.with_(precision=W.FP32)
    g = gpu_leg(H, s32, bank, step)
    fp32_check(g, o, name, fp32_without(H, orc, s32, bank, step, lambda skip: orc.mc_leg(spec, step, bank, skip=skip)))
    s = g["stats"]
    tot = s["w_absorbed"] + s["w_leaked"] + s["w_census"] + s["w_handoff"] + s["w_killed"]
    assert math.isclose(s["w_source"], tot, rel_tol=1e-5)


# ------------------------------------------------------------------------------------------------
# collided S_N-DG and remap
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("layout", [1, 2])
@pytest.mark.parametrize("order,n", [(4, 35), (8, 40), (8, 7)])
def test_collided_solve_parity(H, orc, order, n, layout):
    """FP64 collided stage against the oracle, on the padded-mesh layout (1, with the cell-solve
    table) and the wavefront layout (2) of the sweep."""
    spec = W.checkerboard(n_s=1, n_hist=20_000, cells_per_block=max(1, n // 7)).with_(sn_order=order, sn_tol=1e-13,
                                                                                      sn_layout=layout)
    bank = W.random_bank(spec, 4000, seed=3)
    o = orc.mc_leg(spec, 0, bank, elem=orc.SERIES)
    phi_o, it_o = orc.sn_solve(spec, o["mom"])
    g = gpu_leg(H, spec, bank, 0)
    st = g["P"].collided_solve()
    phi_g = g["P"].tally("sn_phi")
    scale = np.max(np.abs(phi_o[:, 0]))
    assert abs(st["sn_iterations"] - it_o) <= 1
    assert np.allclose(phi_g, phi_o, rtol=1e-9, atol=1e-10 * scale)


@pytest.mark.parametrize("layout", [1, 2])
@pytest.mark.parametrize("order", [4, 8])
def test_collided_solve_fp32(H, orc, order, layout):
    """FP32 collided stage: the GPU's own hand-off moments solved by the FP64 oracle; cells above
    1e-3 of the peak agree within 1e-4 relative (stop test at 2e-6 relative change)."""
    spec = W.checkerboard(n_s=1, n_hist=20_000, cells_per_block=5, precision=W.FP32).with_(sn_order=order,
                                                                                          sn_tol=1e-7,
                                                                                          sn_layout=layout)
    bank = W.random_bank(spec, 4000, seed=5)
    g = gpu_leg(H, spec, bank, 0)
    g["P"].collided_solve()
    phi_g = g["P"].tally("sn_phi")
    phi_o, _ = orc.sn_solve(spec.with_(precision=W.FP64, sn_tol=1e-13), g["mom"])
    peak = np.max(np.abs(phi_o[:, 0]))
    sel = np.abs(phi_o[:, 0]) >= 1e-3 * peak
    err = np.max(np.abs(phi_g[sel, 0] - phi_o[sel, 0]) / np.abs(phi_o[sel, 0]))
    print(f"\nFP32 collided S{order}: max rel err of phi_0 on resolved cells {err:.2e}")
    assert err < 1e-4
    assert np.allclose(phi_g[:, 1:], phi_o[:, 1:], rtol=0, atol=1e-4 * peak)


@pytest.mark.parametrize("layout", [1, 2])
@pytest.mark.parametrize("prec", [W.FP64, W.FP32])
def test_collided_solve_tall_mesh(H, orc, prec, layout):
    """8 x 700 cells: 22 row strips for at most 16 warps, so strip-to-strip ring slots are reused."""
    n = 8
    sa = np.full(n * 700, 0.2)
    ss = np.full(n * 700, 0.8)
    spec = W.ProblemSpec(nx=n, ny=700, lx=1.0, ly=87.5, sigma_a=sa, sigma_s=ss, Q=np.ones(n * 700), c=1.0, dt=0.5,
                         n_s=0, n_hist=20_000, seed=2, precision=prec, sn_order=8, sn_tol=1e-13 if prec == W.FP64 else 1e-7,
                         sn_layout=layout)
    g = gpu_leg(H, spec, None, 0)
    g["P"].collided_solve()
    phi_g = g["P"].tally("sn_phi")
    phi_o, _ = orc.sn_solve(spec.with_(precision=W.FP64, sn_tol=1e-13), g["mom"])
    scale = np.max(np.abs(phi_o[:, 0]))
    if prec == W.FP64:
        assert np.allclose(phi_g, phi_o, rtol=1e-9, atol=1e-10 * scale)
    else:
        assert np.allclose(phi_g, phi_o, rtol=1e-4, atol=1e-5 * scale)


@pytest.mark.parametrize("prec", [W.FP64, W.FP32])
def test_sweep_layouts_agree(H, prec):
    """The two memory layouts of the sweep (padded mesh, wavefront order) run the same arithmetic in
    the same order: the collided flux agrees to rounding (FP32: bit for bit expected; FP64: the
    padded mesh takes the tabulated cell solve), on a mesh with a ragged last strip and ragged
    columns."""
    base = W.checkerboard(n_s=1, n_hist=20_000, cells_per_block=3, precision=prec)
    base = base.with_(nx=37, ny=45, sigma_a=np.resize(base.sigma_a, 37 * 45), sigma_s=np.resize(base.sigma_s, 37 * 45),
                      Q=np.resize(base.Q, 37 * 45), ic=None, sn_tol=1e-13 if prec == W.FP64 else 1e-7)
    bank = W.random_bank(base, 3000, seed=4)
    out = {}
    for layout in (1, 2):
        P = H.Problem(base.with_(sn_layout=layout))
        P.set_bank(bank)
        P.set_step(0)
        P.mc_leg()
        st = P.collided_solve()
        out[layout] = (P.tally("sn_phi"), st["sn_iterations"])
        P.close()
    a, b = out[1][0], out[2][0]
    scale = np.max(np.abs(a[:, 0]))
    print(f"\nlayouts: iterations {out[1][1]} / {out[2][1]}, bitwise equal: {np.array_equal(a, b)}")
    assert out[1][1] == out[2][1]
    assert np.allclose(a, b, rtol=0, atol=(1e-12 if prec == W.FP64 else 1e-6) * scale)


def test_sweep_layout_validation(H):
    spec = W.checkerboard(n_s=1, n_hist=1000, cells_per_block=1)
    with pytest.raises(H.HybError):
        H.Problem(spec.with_(sn_layout=3))


@pytest.mark.parametrize("cap,order", [(0, 0), (10 ** 7, 0), (0, 1), (10 ** 7, 1), (9000, 1), (0, 2), (10 ** 7, 2),
                                       (9000, 2)])
def test_remap_parity(H, orc, cap, order):
    """The remap's census against the oracle: comb or not, slot order or cell order (a stable
    sort by cell before the comb), element by element."""
    spec = W.checkerboard(n_s=2, n_hist=20_000, cells_per_block=4).with_(census_cap=cap, census_order=order)
    bank = W.random_bank(spec, 15_000, seed=8)
    o = orc.mc_leg(spec, 2, bank, elem=orc.SERIES)
    phi_o, _ = orc.sn_solve(spec, o["mom"])
    ob, ost, ocomb = orc.remap(spec, 2, bank, o["pre"], o["post"], phi_o, elem=orc.SERIES)
    g = gpu_leg(H, spec, bank, 2)
    P = g["P"]
    P.set_sn_phi(phi_o)
    rs = P.remap()
    gb = P.bank()
    assert bool(rs["combed"]) == ocomb
    assert gb["n"] == ob["n"]
    assert np.array_equal(gb["cell"], ob["cell"])
    d = spec.lx / spec.nx
    for k in ("fx", "fy"):
        assert np.allclose(gb[k], ob[k], rtol=0, atol=1e-10 * d), k
    for k in ("ox", "oy"):
        assert np.allclose(gb[k], ob[k], rtol=0, atol=1e-12), k
    assert np.allclose(gb["w"], ob["w"], rtol=1e-10, atol=0)
    assert rs["histories"] == ost["histories"] and rs["leaked"] == ost["leaked"]
    assert math.isclose(rs["w_source"], ost["w_source"], rel_tol=1e-10)
    for k in ("w_absorbed", "w_leaked", "w_killed"):
        assert math.isclose(rs[k], ost[k], rel_tol=1e-10, abs_tol=1e-12 * ost["w_source"]), (k, rs[k], ost[k])


@pytest.mark.parametrize("prec,order,sampler,limits", [(W.FP64, 0, W.SOBOL, 0), (W.FP32, 0, W.SOBOL, 0),
                                                       (W.FP64, 1, W.SOBOL, 0), (W.FP64, 1, W.HALTON, 0),
                                                       (W.FP64, 0, W.SOBOL, 1), (W.FP64, 2, W.SOBOL, 0),
                                                       (W.FP32, 2, W.SOBOL, 0)])
def test_multistep_hybrid(H, orc, prec, order, sampler, limits):
    spec = W.pulse(n_hist=8192).with_(precision=prec, sn_tol=1e-12 if prec == W.FP64 else 1e-7, census_order=order,
                                      sampler=sampler)
    if limits:   # space-dependent N_s: limit 2 in the left half, 0 in the right half
        spec = spec.with_(n_s=2, n_s_cell=np.where(np.arange(spec.ncells) % spec.nx < spec.nx // 2, 2, 0))
    ospec = spec.with_(precision=W.FP64, sn_tol=1e-12)
    P = H.Problem(spec)
    # FP64: the oracle on the FP64 path's own map recipe (whole-particle comb decisions must agree);
    # FP32: the libm maps
    el = orc.SERIES if prec == W.FP64 else orc.LIBM
    ob = orc.init_bank(ospec, ospec.ic, elem=el)
    errs, tot = [], []
    for k in range(4):
        stats = P.step(1)[0]
        r = orc.step(ospec, k, ob, elem=el)
        ob = r["bank"]
        flux_g = P.tally("flux")
        peak = np.max(np.abs(r["flux"]))
        sel = np.abs(r["flux"]) >= 1e-3 * peak
        err = float(np.max(np.abs(flux_g[sel] - r["flux"][sel]) / np.abs(r["flux"][sel])))
        errs.append(err)
        tot.append(abs(flux_g.sum() / r["flux"].sum() - 1.0))
        assert stats["bank_size"] == ob["n"]
    print(f"\nmulti-step flux max rel err per step ({'FP64' if prec else 'FP32'}): {errs}, total {tot}")
    if prec == W.FP64:
        assert max(errs) < 1e-9
    else:
        # FP32 trajectories diverge from the FP64 oracle by whole-particle decisions (comb teeth,
        # near-tie crossings) after the first remap; the step totals must still agree closely
        assert max(tot) < 1e-4 and max(errs) < 2e-2


# ------------------------------------------------------------------------------------------------
# full-size configurations
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n_s", [0, 1, 2, 4])
def test_checkerboard_full_size_leg(H, orc, opool, n_s):
    """112x112 checkerboard, 10^6 source histories + a 10^6 bank (the benchmark leg, in the launch
    configuration the benchmark times): FP64 against both oracle modes, FP32 against the libm one."""
    spec = W.checkerboard(n_s=n_s, n_hist=1_000_000)
    bank = W.random_bank(spec, 1_000_000, seed=n_s)
    g = gpu_leg(H, spec, bank, 1)
    o = opool.mc_leg(spec, 1, bank, want_hist=True, elem=orc.SERIES)
    mism = int(np.sum(np.any(g["hist"] != o["hist"], axis=1)))
    assert mism == 0, mism
    check_counts(g["stats"], o["stats"])
    check_fp64_tallies(g, o)
    ol = opool.mc_leg(spec, 1, bank, want_hist=True, want_margin=True, elem=orc.LIBM)
    check_fp64_libm(g, ol, spec, bank, f"checkerboard N_s={n_s}")
    s32 = spec.with_(precision=W.FP32)
    g32 = gpu_leg(H, s32, bank, 1)
    fp32_check(g32, ol, f"checkerboard N_s={n_s}",
               fp32_without(H, orc, s32, bank, 1, lambda skip: opool.mc_leg(spec, 1, bank, skip=skip)))


def test_large_diffusive_subsample(H, orc, opool):
    """1024x1024 diffusive mesh (sigma_t in {1, 10, 1000}, ratio 0.999 in the thick blocks), N_s = 8
    (29 point dimensions): the 1/16 subsample of its 10^8-history step -- the first 6.25e6 source
    births (a prefix of the Sobol set) and an injected census bank of 6.25e6 particles -- in the
    leg's full launch configuration. FP64 against both oracle modes (records, counters, tallies),
    FP32 at the FP32 bar."""
    n = 6_250_000
    spec = W.large(n=1024, n_hist=n, precision=W.FP64)
    bank = W.random_bank(spec, n, seed=4)
    g = gpu_leg(H, spec, bank, 3)
    o = opool.mc_leg(spec, 3, bank, want_hist=True, elem=orc.SERIES)
    mism = int(np.sum(np.any(g["hist"] != o["hist"], axis=1)))
    assert mism == 0, mism
    check_counts(g["stats"], o["stats"])
    check_fp64_tallies(g, o)
    del o
    ol = opool.mc_leg(spec, 3, bank, want_hist=True, want_margin=True, elem=orc.LIBM)
    check_fp64_libm(g, ol, spec, bank, "large 1024^2 subsample")
    del g
    s32 = spec.with_(precision=W.FP32)
    g32 = gpu_leg(H, s32, bank, 3)
    fp32_check(g32, ol, "large 1024^2 subsample",
               fp32_without(H, orc, s32, bank, 3, lambda skip: opool.mc_leg(spec, 3, bank, skip=skip)),
               rtol=FP32_RTOL_THICK)
    s = g32["stats"]
    tot = s["w_absorbed"] + s["w_leaked"] + s["w_census"] + s["w_handoff"] + s["w_killed"]
    assert math.isclose(s["w_source"], tot, rel_tol=1e-5)


@pytest.mark.parametrize("order", [0, 1, 2])
def test_ns_infinity_pure_mc(H, orc, order):
    """N_s = infinity (pure (Q)MC, no hand-off, no collided stage): the MC-leg census survivors,
    combed to census_cap, are the next bank. Three steps of a pulse (bank only) and of a small
    checkerboard (bank + births) against the oracle: banks cell for cell, fluxes to rounding."""
    for spec, bank0 in ((W.pulse(n_hist=4096), None),
                        (W.checkerboard(n_s=0, n_hist=6000, cells_per_block=2), None)):
        spec = spec.with_(n_s=W.NS_INF, precision=W.FP64, census_order=order)
        P = H.Problem(spec)
        ob = orc.init_bank(spec, spec.ic, elem=orc.SERIES) if spec.ic is not None else None
        for k in range(3):
            st = P.step(1)[0]
            r = orc.step(spec, k, ob, elem=orc.SERIES)
            ob = r["bank"]
            gb = P.bank()
            assert st["sn_iterations"] == 0
            assert gb["n"] == ob["n"], (spec.name, k)
            assert np.array_equal(gb["cell"], ob["cell"]), (spec.name, k)
            for q in ("fx", "fy", "ox", "oy"):
                assert np.allclose(gb[q], ob[q], rtol=0, atol=1e-12 * max(spec.lx, 1.0)), (spec.name, k, q)
            assert np.allclose(gb["w"], ob["w"], rtol=1e-10, atol=0), (spec.name, k)
            f = P.tally("flux")
            assert np.allclose(f, r["flux"], rtol=1e-9, atol=1e-12 * np.max(np.abs(r["flux"]))), (spec.name, k)
        P.close()


@pytest.mark.parametrize("prec", [W.FP64, W.FP32])
def test_collided_solve_anderson(H, orc, prec):
    """Anderson-accelerated source iteration on a diffusive problem (effective scattering ratio
    ~0.9): the same fixed point as the oracle's plain iteration, in fewer sweeps."""
    base = W.checkerboard(n_s=1, n_hist=20_000, cells_per_block=4)
    spec = base.with_(sigma_a=base.sigma_a * 10, sigma_s=base.sigma_s * 10, dt=1.0, sn_order=4,
                      precision=prec, sn_tol=1e-12 if prec == W.FP64 else 1e-7, sn_max_iter=2000)
    bank = W.random_bank(spec, 4000, seed=9)
    g = gpu_leg(H, spec, bank, 0)
    phi_o, it_o = orc.sn_solve(spec.with_(precision=W.FP64, sn_tol=1e-13, sn_max_iter=5000), g["mom"])
    iters = {}
    for depth in (0, 4):
        P = H.Problem(spec.with_(sn_accel=depth, ic=None))
        P.set_bank(bank)
        P.set_step(0)
        P.mc_leg()
        st = P.collided_solve()
        iters[depth] = st["sn_iterations"]
        phi_g = P.tally("sn_phi")
        scale = np.max(np.abs(phi_o[:, 0]))
        tol = 1e-8 if prec == W.FP64 else 2e-4
        assert np.allclose(phi_g, phi_o, rtol=0, atol=tol * scale), (depth, np.max(np.abs(phi_g - phi_o)) / scale)
        P.close()
    print(f"\nSI iterations plain {iters[0]} (oracle {it_o}), Anderson(4) {iters[4]}")
    assert iters[4] < iters[0] / 2


@pytest.mark.parametrize("order", [0, 1])
def test_additive_remap_variant(H, orc, order):
    """Steps 3'/4' of the previous hybrids (Eq. (R')): the census is the MC leg's census followed
    by the survivors of births from sigma_s (phi_post + phi_c). FP64 against the oracle over three
    steps (banks cell for cell, fluxes to rounding), with and without a comb."""
    cb = W.checkerboard(n_s=1, n_hist=6000, cells_per_block=2)
    for spec in (W.pulse(n_hist=4096, n_s=1), cb, cb.with_(census_cap=4000)):
        spec = spec.with_(remap_variant=1, precision=W.FP64, census_order=order, sn_tol=1e-12)
        P = H.Problem(spec)
        ob = orc.init_bank(spec, spec.ic, elem=orc.SERIES) if spec.ic is not None else None
        for k in range(3):
            P.step(1)
            r = orc.step(spec, k, ob, elem=orc.SERIES)
            ob = r["bank"]
            gb = P.bank()
            assert gb["n"] == ob["n"], (spec.name, k)
            assert np.array_equal(gb["cell"], ob["cell"]), (spec.name, k)
            for q in ("fx", "fy", "ox", "oy"):
                assert np.allclose(gb[q], ob[q], rtol=0, atol=1e-12 * max(spec.lx, 1.0)), (spec.name, k, q)
            assert np.allclose(gb["w"], ob["w"], rtol=1e-9, atol=0), (spec.name, k)
            f = P.tally("flux")
            assert np.allclose(f, r["flux"], rtol=1e-9, atol=1e-12 * np.max(np.abs(r["flux"]))), (spec.name, k)
        P.close()


def test_additive_remap_variant_fp32(H, orc):
    """The FP32 path of steps 3'/4': step totals close to the FP64 oracle's."""
    spec = W.checkerboard(n_s=1, n_hist=20_000, cells_per_block=2).with_(remap_variant=1, sn_tol=1e-7)
    P = H.Problem(spec.with_(precision=W.FP32))
    ob = None
    for k in range(3):
        P.step(1)
        r = orc.step(spec.with_(precision=W.FP64, sn_tol=1e-12), k, ob)
        ob = r["bank"]
        gb = P.bank()
        assert abs(gb["n"] - ob["n"]) <= max(3, ob["n"] // 1000)
        assert abs(gb["w"].sum() / ob["w"].sum() - 1) < 1e-4
        f = P.tally("flux")
        assert abs(f.sum() / r["flux"].sum() - 1) < 1e-4
    P.close()


def test_remap_variant_validation(H):
    with pytest.raises(H.HybError):   # per-cell limits above n_s
        H.Problem(W.pulse(n_hist=100).with_(n_s=1, n_s_cell=np.full(256, 2, np.int32)))
    with pytest.raises(H.HybError):
        H.Problem(W.pulse(n_hist=100).with_(remap_variant=1, n_s=W.NS_INF))
    with pytest.raises(H.HybError):
        H.Problem(W.pulse(n_hist=100).with_(remap_variant=2))


@pytest.mark.parametrize("where", ["host", "device"])
@pytest.mark.parametrize("prec", [W.FP32, W.FP64])
def test_set_bank_native_equals_set_bank(H, prec, where):
    """A bank given in the problem's own layout (page-locked host arrays: asynchronous copies;
    device arrays: one copy-and-check kernel) steps exactly like the same bank given through the
    checked FP64 host path; an invalid particle in a native upload is reported by the next step."""
    import torch
    spec = W.checkerboard(n_s=2, n_hist=20_000, cells_per_block=2).with_(precision=prec)
    bank = W.random_bank(spec, 5000, seed=3)
    fdt = torch.float32 if prec == W.FP32 else torch.float64
    npdt = np.float32 if prec == W.FP32 else np.float64
    # values representable in the problem precision, so both paths hold the same bank
    for k in ("fx", "fy", "ox", "oy", "w"):
        bank[k] = bank[k].astype(npdt).astype(np.float64)
    A = H.Problem(spec)
    A.set_bank(bank)
    A.step(2)
    B = H.Problem(spec)
    arrs = [torch.from_numpy(bank["cell"].astype(np.int32)).pin_memory()]
    arrs += [torch.from_numpy(bank[k].astype(npdt)).pin_memory() for k in ("fx", "fy", "ox", "oy", "w")]
    if where == "device":
        arrs = [a.cuda() for a in arrs]
    assert arrs[1].dtype == fdt
    B.set_bank_native(*arrs)
    B.step(2)
    assert np.array_equal(A.tally("flux"), B.tally("flux"))
    ba, bb = A.bank(), B.bank()
    assert ba["n"] == bb["n"] and all(np.array_equal(ba[k], bb[k]) for k in ("cell", "fx", "fy", "ox", "oy", "w"))
    bad = [a.clone() for a in arrs]
    bad[1][7] = 1e3                       # an in-cell offset far outside the cell
    B.set_bank_native(*bad)
    with pytest.raises(H.HybError) as e:
        B.step(1)
    assert e.value.status == H.HYB_EINVAL
    B.set_bank_native(*arrs)              # a valid bank clears the report
    B.step(1)
    A.close()
    B.close()
