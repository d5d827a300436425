"""Batched sweep (many channels of uneven size in one launch per step, CUDA graph chunks)
against independent single-channel handles: the same per-node arithmetic, so fields,
residuals and convergence step counts must agree bit for bit."""
import numpy as np
import pytest

import lbm_workloads as WL

pytestmark = pytest.mark.gpu
FIELDS = ("phi", "u", "v", "T", "dp")


@pytest.fixture(scope="module")
def pkg():
    import paper_2210_07501_gb300 as p
    p.build()
    p.load()
    return p


def small_sweep(n=7, seed=5):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        nx = int(rng.choice([64, 100, 300, 520]))
        ny = int(rng.choice([17, 24, 40]))
        ab = float(rng.uniform(0.5, 2.0))
        out.append(WL.channel(nx, ny, round(ny / (1 + ab)), W=4.0, sigma1=float(rng.uniform(-2e-4, 2e-4)),
                              sigma2=float(rng.uniform(-4e-3, 0.0)), cond_ratio=float(rng.uniform(0.5, 3.0)),
                              visc_ratio=float(rng.uniform(0.5, 3.0)), tau_flow=1.0, tau_T=1.4))
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_single_handles(pkg, precision):
    ws = small_sweep()
    b = pkg.LbmBatch(ws, precision=precision)
    b.lbm_batch_set_check_interval(50)
    rows = b.lbm_batch_autotune(2)
    assert rows > 0
    b.lbm_batch_step(300)
    for c, w in enumerate(ws):
        g = pkg.Lbm(w["domain"], w["params"], precision=precision)
        g.lbm_set_check_interval(50)
        g.lbm_step(300)
        a, r = b.lbm_batch_fields(c), g.lbm_fields()
        for k in FIELDS:
            assert np.array_equal(a[k], r[k]), (c, k)
        d = g.lbm_diag()
        assert b.lbm_batch_diag(c)["residual"] == pytest.approx(d["residual"], rel=1e-12)
        g.close()
    b.close()


def test_batch_run_to_steady_matches_single(pkg):
    ws = small_sweep(n=5, seed=9)
    tol, K = 1e-6, 100
    b = pkg.LbmBatch(ws, precision="fp32")
    b.lbm_batch_set_check_interval(K)
    steps, conv = b.lbm_batch_run_to_steady(tol, 40000)
    assert sum(conv) >= 2
    for c, w in enumerate(ws):
        g = pkg.Lbm(w["domain"], w["params"], precision="fp32")
        g.lbm_set_check_interval(K)
        ok, n = g.lbm_run_to_steady(tol, 40000)
        assert ok == conv[c] and n == steps[c], (c, ok, conv[c], n, steps[c])
        a, r = b.lbm_batch_fields(c), g.lbm_fields()
        for k in FIELDS:
            assert np.array_equal(a[k], r[k]), (c, k)
        g.close()
    assert len(set(steps)) > 1      # uneven channels converge at different times
    b.close()
