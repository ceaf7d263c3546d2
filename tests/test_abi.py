"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports every entry point
that include/hyb.h declares, and its host-side tables and validation behave."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2511_16821_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hyb():
    from paper_2511_16821_gb300 import build, hyb as H
    build.build()
    return H


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "hyb.h")).read()
    return sorted(set(re.findall(r"HYB_API\s+[\w\s\*]+?\b(hyb_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(hyb):
    syms = declared_symbols()
    assert len(syms) >= 20
    L = C.CDLL(hyb.lib()._name)
    for s in syms:
        assert hasattr(L, s), s


def test_sobol_table_matches_oracle(hyb, orc):
    assert np.array_equal(hyb.sobol_table(65), orc.sobol_table(65))


@pytest.mark.parametrize("order", [4, 8])
def test_quadrature_matches_oracle(hyb, orc, order):
    ox, oy, w = hyb.quadrature(order)
    a, b, _, c = orc.quadrature(order)
    assert np.allclose(ox, a, atol=1e-14) and np.allclose(oy, b, atol=1e-14)
    assert np.allclose(w, c, rtol=1e-13)


def _bad(spec, **kw):
    return spec.with_(**kw)


@pytest.mark.parametrize("mut", [
    dict(nx=0), dict(ny=5000), dict(dt=0.0), dict(c=-1.0), dict(n_s=-1), dict(sn_order=6),
    dict(n_hist=0), dict(sampler=7), dict(precision=3), dict(w_min=1.5), dict(sn_max_iter=0),
    dict(sn_layout=3), dict(sn_layout=-1), dict(seg_limit=-1), dict(seg_limit=(1 << 30) + 1), dict(wait_limit=-5),
    dict(tally_copies=-1), dict(tally_copies=65), dict(sort_every=-1), dict(leg_sort_every=-1), dict(priv_tile=-2),
    dict(priv_tile=33), dict(census_order=1, remap_variant=1, census_cap=(1 << 31) - 1, n_hist=(1 << 31) - 1),
])
def test_workspace_size_rejects_bad_descriptors(hyb, mut):
    spec = W.pulse(n_hist=100)
    if "nx" in mut or "ny" in mut:
        n = mut.get("nx", spec.nx) * mut.get("ny", spec.ny)
        spec = spec.with_(sigma_a=np.ones(max(n, 1)), sigma_s=np.ones(max(n, 1)), ic=None)
    with pytest.raises(hyb.HybError) as e:
        hyb.workspace_size(spec.with_(**mut))
    assert e.value.status == hyb.HYB_EINVAL


@pytest.mark.parametrize("field", ["sigma_a", "sigma_s", "Q"])
def test_rejects_nonfinite_or_negative_data(hyb, field):
    spec = W.homogeneous(n=4, Q=1.0)
    for bad in (np.nan, -1.0, np.inf):
        arr = np.array(getattr(spec, field), dtype=float)
        arr[3] = bad
        with pytest.raises(hyb.HybError):
            hyb.workspace_size(spec.with_(**{field: arr}))


def test_workspace_size_scales_with_histories(hyb):
    a = hyb.workspace_size(W.checkerboard(n_hist=10_000))
    b = hyb.workspace_size(W.checkerboard(n_hist=1_000_000))
    c = hyb.workspace_size(W.checkerboard(n_hist=1_000_000, precision=W.FP32))
    assert a < b and c < b


def _sweep_bytes(nx, ny, nord, fp64, wave):
    """The collided solve's sweep buffers as the layouts define them: sources (4 + 1 values per
    entry) and per-ordinate psi (4 per entry), plus the FP64 cell-solve table (9 per ordinate
    class and entry, padded mesh only, at most 8 strips and 64 MB)."""
    T = 8 if fp64 else 4
    PF = 4 if fp64 else 8
    nstrip = (ny + 31) // 32
    if wave:
        nt = (nx + 31 + PF - 1) // PF * PF + PF
        ent = nstrip * nt * 32
        return 4 * ent * 5 * T + nord * ent * 4 * T
    plane = (ny + 1) * (nx + 2 * (32 + 2 * PF))
    tab = (nord // 4) * plane * 9 * T if fp64 and nstrip <= 8 else 0
    tab = tab if tab <= 64 << 20 else 0
    return plane * 5 * T + nord * nx * ny * 4 * T + tab


@pytest.mark.parametrize("prec", [W.FP64, W.FP32])
def test_workspace_size_by_sweep_layout(hyb, prec):
    """Host-side layout choice: the workspaces of the padded-mesh (1) and wavefront (2) layouts
    differ by exactly the difference of their sweep buffers (to the 256-byte alignment of the
    workspace's parts), and the automatic choice (0) keeps the padded mesh on the 112^2 benchmark
    mesh and takes the wavefront order on the 1024^2 mesh (per-ordinate solutions above 48 MB)."""
    spec = W.checkerboard(n_hist=10_000, precision=prec)
    fp64 = prec == W.FP64
    ws = {L: hyb.workspace_size(spec.with_(sn_layout=L)) for L in (0, 1, 2)}
    want = _sweep_bytes(112, 112, 40, fp64, True) - _sweep_bytes(112, 112, 40, fp64, False)
    assert abs((ws[2] - ws[1]) - want) <= 3 * 256
    assert ws[0] == ws[1]
    big = W.large(n=1024, n_hist=10_000, precision=prec)
    wb = {L: hyb.workspace_size(big.with_(sn_layout=L)) for L in (0, 1, 2)}
    assert wb[0] == wb[2]
    want_b = _sweep_bytes(1024, 1024, 40, fp64, True) - _sweep_bytes(1024, 1024, 40, fp64, False)
    assert abs((wb[2] - wb[1]) - want_b) <= 3 * 256


def test_no_cpu_fallback_without_gpu(hyb):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        hyb.Problem(W.pulse(n_hist=10))


def test_input_generators_are_deterministic():
    a = W.random_batch_problem(0, 5)
    b = W.random_batch_problem(0, 5)
    assert a.nx == b.nx and np.array_equal(a.sigma_a, b.sigma_a) and a.n_hist == b.n_hist
    c = W.checkerboard(cells_per_block=4)
    assert c.nx == 28 and c.Q.sum() == 16 and c.sigma_s.reshape(28, 28)[13, 13] == 1.0
    big = W.large(n=64, block=8, n_hist=10)
    assert set(np.round(big.sigma_a + big.sigma_s, 6)) <= {1.0, 10.0, 1000.0}


def test_descriptor_layout_matches_header(hyb):
    # the binding's descriptor struct has the header's size (fields appended at the end keep the
    # 8-byte alignment of the C struct)
    assert C.sizeof(hyb.Desc) % 8 == 0
    names = [f for f, _ in hyb.Desc._fields_]
    txt = open(os.path.join(ROOT, "include", "hyb.h")).read()
    body = txt[txt.index("typedef struct {\n    int32_t nx, ny;"):txt.index("} hyb_problem_desc;")]
    for n in ("seg_limit", "wait_limit", "sn_layout", "n_s_cell", "tally_copies", "sort_every", "leg_sort_every",
              "priv_tile"):
        assert n in names and n in body
    # the binding's fields follow the header's order
    order = [n for n in names if not n.startswith("pad")]
    pos = [body.index(" " + n + ";") if (" " + n + ";") in body else body.index(n) for n in order]
    assert pos == sorted(pos)


def test_workspace_size_by_leg_options(hyb):
    """The phased leg adds two buffers of saved histories (48 B each in FP32) and their sort; the
    copies of the tally arrays scale the tally storage; the shared-memory window adds nothing."""
    spec = W.checkerboard(n_s=2, n_hist=10_000, cells_per_block=4).with_(precision=W.FP32)
    base = hyb.workspace_size(spec)
    cap = 10_000 + 10_000                       # bank capacity + births
    assert hyb.workspace_size(spec.with_(leg_sort_every=4)) - base >= 2 * cap * 48 + 2 * cap * 8
    assert hyb.workspace_size(spec.with_(priv_tile=16)) == base == hyb.workspace_size(spec.with_(priv_tile=0))
    nc = spec.nx * spec.ny
    grow = hyb.workspace_size(spec.with_(tally_copies=8)) - hyb.workspace_size(spec.with_(tally_copies=1))
    assert abs(grow - 7 * 6 * nc * 8) <= 3 * 256   # each array 256-byte aligned


def test_tuning_spaces():
    from paper_2511_16821_gb300 import autotune
    # the batch's space: the named values replace the defaults, the rest keep them
    c = autotune.candidates({"block": (256,), "chunk": (2048,)})
    assert len(c) == len(autotune.DEFAULT_SPACE["streams"]) * len(autotune.DEFAULT_SPACE["ctas_per_sm"])
    assert all(x["block"] == 256 and x["chunk"] == 2048 for x in c)
    # one problem's space: every combination of the named knobs, nothing else
    c = autotune.candidates({"tally_copies": (1, 4), "priv_tile": (0, 16)}, {})
    assert sorted((x["tally_copies"], x["priv_tile"]) for x in c) == [(1, 0), (1, 16), (4, 0), (4, 16)]
    assert all(set(x) == {"tally_copies", "priv_tile"} for x in c)
    n = 1
    for v in autotune.PROBLEM_SPACE.values():
        n *= len(v)
    assert len(autotune.candidates(None, autotune.PROBLEM_SPACE)) == n


def test_priv_window_choice(hyb):
    """The leg's shared-memory window: the densest square of the source (the checkerboard's
    source block, cells 48..63 of 112), automatic only at N_s = 0 with a concentrated source."""
    cb0 = W.checkerboard(n_s=0, n_hist=1000)
    assert hyb.priv_window(cb0) == (48, 48, 16)                      # automatic (the default, -1)
    assert hyb.priv_window(cb0.with_(priv_tile=0)) == (0, 0, 0)
    x0, y0, s = hyb.priv_window(cb0.with_(priv_tile=8))              # inside the block
    assert s == 8 and 48 <= x0 <= 56 and 48 <= y0 <= 56
    assert hyb.priv_window(W.checkerboard(n_s=2, n_hist=1000))[2] == 0   # N_s >= 1: none by default
    assert hyb.priv_window(W.checkerboard(n_s=2, n_hist=1000).with_(priv_tile=16)) == (48, 48, 16)
    uni = W.homogeneous(n=32, Q=1.0, n_s=0)
    assert hyb.priv_window(uni)[2] == 0                              # spread source: none
    assert hyb.priv_window(W.homogeneous(n=12, Q=1.0, n_s=0).with_(priv_tile=16)) == (0, 0, 12)   # at most the mesh
