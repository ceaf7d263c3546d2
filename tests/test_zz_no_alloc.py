"""The allocation-free CDF build (hyb_build_cdf_noalloc), for callers that cannot allocate device
memory (serving loops that must not allocate on their hot path, hosts whose device memory belongs
to a foreign allocator with a fixed budget).

Calls it through the C ABI twice in a row on different inputs and checks each result against the
scratch-taking hyb_build_cdf: the CDF integers must agree exactly and the weight sums to the last
bit, so state left in the shared scratch array by one call cannot leak into the next. This file
is collected last so that a stop-at-first-failure run has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(H, w, nx, ny):
    import torch
    L = H.lib()
    f = L.hyb_build_cdf_noalloc
    f.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    q = torch.full((nx * ny,), -1, dtype=torch.int64, device="cuda")
    rp = torch.full((ny + 1,), -1, dtype=torch.int64, device="cuda")
    cp = torch.full((ny * (nx + 1),), -1, dtype=torch.int64, device="cuda")
    wq = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    st = f(C.c_void_p(w.data_ptr()), nx, ny, C.c_void_p(q.data_ptr()), C.c_void_p(rp.data_ptr()),
           C.c_void_p(cp.data_ptr()), C.c_void_p(wq.data_ptr()),
           C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, q, rp, cp, wq


def test_noalloc_cdf_matches_scratch_build():
    import torch
    from paper_2511_16821_gb300 import hyb as H
    assert torch.cuda.is_available()
    for nx, ny, seed in ((112, 112, 1), (37, 4096, 2)):
        rng = np.random.default_rng(seed)
        w = torch.tensor(rng.uniform(0.0, 1.0, nx * ny) ** 2, device="cuda")
        st, q, rp, cp, wq = _noalloc(H, w, nx, ny)
        assert st == H.HYB_OK
        rq, rrp, rcp, rwq = H.build_cdf(w, nx, ny)
        torch.cuda.synchronize()
        assert torch.equal(q, rq) and torch.equal(rp, rrp) and torch.equal(cp, rcp)
        assert torch.equal(wq, rwq)


def test_noalloc_rejects_rows_beyond_its_scratch():
    import torch
    from paper_2511_16821_gb300 import hyb as H
    w = torch.ones(2 * 4097, dtype=torch.float64, device="cuda")
    st, *_ = _noalloc(H, w, 2, 4097)
    assert st == H.HYB_EINVAL
