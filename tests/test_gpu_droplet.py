"""The paper's droplet workloads on the GPU path (Sec. 5.1 and Laplace's law).

* Parity: the drop-migration case (160 x 320, D2Q9 for all three lattices, a curved
  interface in every direction, a ragged second strip) against the FP64 oracle; FP64 bars
  from the oracle's own FMA sensitivity on this case (as in test_gpu_parity), FP32 bars
  stated from the measured errors.
* Laplace's law on the GPU: p_in - p_out = sigma / R for three radii (the oracle's own pin
  covers one radius on the CPU).
* Migration: the drop moves up the temperature gradient (towards lower sigma) at about
  0.8 U_YGB, the value the paper and other 2-D computations report.
"""
import os

import numpy as np
import pytest

import lbm_workloads as WL

pytestmark = pytest.mark.gpu
FIELDS = ("phi", "u", "v", "T", "dp")


def rel_l2(a, b):
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    oracle.build(fma=True)
    oracle.set_threads(os.cpu_count() or 1)
    return oracle


def drop_case():
    w = WL.workload("paper-drop-migration-160x320")
    d, p = w["domain"], w["params"]
    init = WL.drop_fields(d["nx"], d["ny"], WL.DROP_RADIUS, d["W"], p["T_hot"], p["T_cold"])
    return w, init


def oracle_fields(orc, w, init, steps, fma=False):
    o = orc.Oracle(w["domain"], w["params"], fma=fma)
    o.init(**init)
    o.step(steps)
    f = o.fields()
    o.close()
    return f


def gpu_fields(w, init, steps, precision):
    from paper_2210_07501_gb300 import Lbm
    g = Lbm(w["domain"], w["params"], precision=precision)
    g.lbm_init_fields(**init)
    g.lbm_step(steps)
    f = g.lbm_fields()
    g.close()
    return f


def test_drop_case_parity_fp64(orc):
    w, init = drop_case()
    steps = 300
    a = gpu_fields(w, init, steps, "fp64")
    b = oracle_fields(orc, w, init, steps)
    c = oracle_fields(orc, w, init, steps, fma=True)
    for k in FIELDS:
        S = rel_l2(c[k], b[k])
        err = rel_l2(a[k], b[k])
        assert err <= max(1e-12, 10 * S), (k, err, S)


def test_drop_case_parity_fp32(orc):
    w, init = drop_case()
    steps = 300
    a = gpu_fields(w, init, steps, "fp32")
    b = oracle_fields(orc, w, init, steps)
    # measured: phi ~1e-6, T ~1e-7, u, v ~1e-3, dp ~1e-4 (rel. L2; u, v ~1e-5 of the
    # sound speed after 300 steps, so FP32 storage round-off is a visible share of them)
    bars = {"phi": 1e-5, "T": 1e-6, "u": 2e-2, "v": 2e-2, "dp": 5e-3}
    for k in FIELDS:
        assert rel_l2(a[k], b[k]) <= bars[k], (k, rel_l2(a[k], b[k]))


def test_laplace_law_three_radii():
    from paper_2210_07501_gb300 import droplet
    sigma = 1e-3
    res = [droplet.laplace(96, R, sigma, W=4.0, steps=6000) for R in (12.0, 18.0, 24.0)]
    ratios = [r["ratio"] for r in res]
    print("Laplace p_jump R / sigma:", ratios)
    for r in res:
        assert 0.85 <= r["ratio"] <= 1.05, r      # diffuse interface: a few % below 1 at W = 4
        assert r["u_max"] < 1e-5                  # spurious currents stay small
    assert max(ratios) - min(ratios) < 0.06


@pytest.mark.timeout(600)
def test_drop_migrates_at_about_0p8_ygb():
    from paper_2210_07501_gb300 import droplet
    w = WL.workload("paper-drop-migration-160x320")
    r = droplet.migration(w, WL.DROP_RADIUS, t_star_end=2.0, samples=40, precision="fp64")
    u = r["U_over_U_ygb"]
    print("U/U_YGB at t* = 0.5, 1, 1.5, 2:", [float(u[int(len(u) * f) - 1]) for f in (0.25, 0.5, 0.75, 1.0)])
    assert abs(r["U_ygb"] - 1.333e-4) < 1e-6              # the paper's printed value
    late = u[-5:]
    assert np.all(late > 0)                               # towards the hot wall (lower sigma)
    assert 0.70 <= late.mean() <= 0.90, late              # 2-D drops: ~0.80 U_YGB (Sec. 5.1)
    assert np.ptp(late) < 0.05                            # terminal velocity reached
    assert abs(r["x_c"][-1] - r["x_c"][0]) < 0.5          # no sideways drift
