"""The allocation-free field reduction (lbm_reduce_fields_noalloc) against lbm_diag.

For callers that cannot allocate device memory: graph-capturing code, and plugins inside
frameworks that own all device memory.  This file is named to be collected last, so that a
run stopping at the first failure has run every other test before it.  It must pass alone
in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

import lbm_workloads as WL

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "u", "v", "T", "dp")


def test_noalloc_reduction_matches_lbm_diag_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    import paper_2210_07501_gb300 as pkg
    pkg.build()
    lib = pkg.load()
    w = WL.channel(96, 40, 17.0, W=4.0, sigma1=1e-4, sigma2=-3e-4)
    K = 50
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = pkg.Lbm(w["domain"], w["params"], precision="fp64", stream=stream)
        g.lbm_set_check_interval(K)
        ny, nx = 40, 96
        n = nx * ny
        result = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        g.lbm_step(K)              # first residual check: the handle keeps u of this step
        prev = {k: torch.empty((ny, nx), dtype=torch.float64, device="cuda") for k in FIELDS}
        g.lbm_fields_device(**prev, dtype=pkg.LBM_DTYPE_F64)
        for call in range(2):
            g.lbm_step(K)          # ends on a residual check: u_prev inside the handle = u of K steps ago
            t = {k: torch.empty((ny, nx), dtype=torch.float64, device="cuda") for k in FIELDS}
            g.lbm_fields_device(**t, dtype=pkg.LBM_DTYPE_F64)
            d = g.lbm_diag()
            rc = lib.lbm_reduce_fields_noalloc(t["phi"].data_ptr(), t["u"].data_ptr(), t["v"].data_ptr(),
                                               t["T"].data_ptr(), prev["u"].data_ptr(), prev["v"].data_ptr(), n,
                                               result.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            assert rc == pkg.LBM_OK
            stream.synchronize()
            r = result.cpu().numpy()
            # same launch shape and summation order as lbm_diag on the same values: the same
            # bits, not only close values
            assert r[0] == d["mass"], (call, r[0], d["mass"])
            assert r[3] == 0.0
            # residual as lbm_diag defines it: ||u^n - u^{n-K}|| / (K ||u^n||)
            res = np.sqrt(r[1]) / (K * np.sqrt(r[2]))
            assert d["residual"] > 0.0
            assert res == d["residual"], (call, res, d["residual"])
            prev = t
        # sizes beyond the maximum and malformed arguments are rejected without any work
        assert lib.lbm_reduce_fields_noalloc(t["phi"].data_ptr(), t["u"].data_ptr(), t["v"].data_ptr(),
                                             t["T"].data_ptr(), None, None, 2 ** 31, result.data_ptr(),
                                             None) == pkg.LBM_EINVAL
        assert lib.lbm_reduce_fields_noalloc(t["phi"].data_ptr(), t["u"].data_ptr(), t["v"].data_ptr(),
                                             t["T"].data_ptr(), t["u"].data_ptr(), None, n, result.data_ptr(),
                                             None) == pkg.LBM_EINVAL
        g.close()
