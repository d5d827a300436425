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


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp16"])
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


def closed_form_u_max(c):
    """Interface U_max of the closed-form solution of Sec. 3 (oracle's analytic module), read
    off as the product's trends module reads the LB fields: the mean of the two node rows
    that straddle the interface."""
    from oracle import analytic as A
    d, p = c["domain"], c["params"]
    ch = A.Channel(l=d["nx"] / max(d["heat_periods"], 1), a=d["ny"] - d["b"], b=d["b"], k_ratio=p["cond_ratio"],
                   mu_ratio=p["visc_ratio"], mu_b=(p["tau_flow"] - 0.5) / 3.0, sigma_T=p["sigma1"],
                   sigma_TT=p["sigma2"], T_h=p["T_hot"], T_c=p["T_cold"], T_ref=p["T_ref"], dT=p["dT"])
    x = np.arange(d["nx"], dtype=float)
    u_lo, _ = A.velocity(ch, x, np.full_like(x, -0.5))
    u_hi, _ = A.velocity(ch, x, np.full_like(x, 0.5))
    return float(np.max(np.abs(0.5 * (u_lo + u_hi))))


def test_sweep_to_steady_state_against_closed_form(pkg):
    """The seeded uneven sweep run to steady state in one batch (FP32, residual checks every
    K steps): every channel that reaches the tolerance has an interface velocity within the
    band the diffuse interface allows of the closed-form solution (Sec. 3).  Default: the
    first six 256 x 64 channels of the seeded 96-channel sweep, to r <= 1e-7;
    LBM_SWEEP_FULL=1: the first 16 channels of the seeded 96-channel sweep to r <= 1e-8
    (prints one JSON line)."""
    import json
    import os
    from paper_2210_07501_gb300 import trends
    full = os.environ.get("LBM_SWEEP_FULL") == "1"
    if full:
        cases, tol, K, nmax = WL.sweep_cases(96, seed=0)[:16], 1e-8, 1000, int(os.environ.get("LBM_SWEEP_MAX", "1500000"))
    else:
        cases = [c for c in WL.sweep_cases(96, seed=0) if c["domain"]["nx"] == 256 and c["domain"]["ny"] == 64][:6]
        tol, K, nmax = 1e-7, 100, 600000
    b = pkg.LbmBatch(cases, precision="fp32")
    b.lbm_batch_set_check_interval(K)
    b.lbm_batch_autotune(3)
    import time
    t0 = time.perf_counter()
    steps, conv = b.lbm_batch_run_to_steady(tol, nmax)
    secs = time.perf_counter() - t0
    rows = []
    for c, w in enumerate(cases):
        f = b.lbm_batch_fields(c)
        u_lb = trends.interface_u_max(f["u"], w["domain"]["b"])
        u_cf = closed_form_u_max(w)
        rows.append({"name": w["name"], "nx": w["domain"]["nx"], "ny": w["domain"]["ny"], "steps": int(steps[c]),
                     "converged": bool(conv[c]), "residual": b.lbm_batch_diag(c)["residual"], "U_lb": u_lb,
                     "U_closed_form": u_cf, "ratio": u_lb / u_cf})
    b.close()
    print(json.dumps({"sweep_steady": {"tol": tol, "check_interval": K, "max_steps": nmax, "seconds": secs,
                                       "converged": int(sum(conv)), "cases": len(cases), "rows": rows}}))
    # measured: default, 3 of 6 at r <= 1e-7 within 400k steps (the slow settling of the
    # interface still under way in the others); full, 7 of 16 at r <= 1e-8 within 1.5M steps
    # (the 1024-wide channels settle over ~1e7 steps)
    assert sum(conv) >= (3 if not full else 6)
    for r in rows:
        if r["converged"]:
            # W / b up to 0.33 on these channels: the diffuse interface costs up to ~20 %
            # (measured 0.88 .. 1.03)
            assert 0.75 <= r["ratio"] <= 1.15, r
