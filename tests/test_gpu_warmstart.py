"""The learned warm start against the plain cold start and against a start from the
closed-form temperature of Sec. 3 (the oracle's analytic module, computed here: the
product holds no closed form).  The surrogate is trained with the library's own kernels
on steady channels produced by the batched solver; it sees only the parameters, the
heating profile and the geometry.

Default: a small case (64 x 32 channels, 96 training seeds run to r <= 1e-6, 8 held-out
seeds run to r <= 1e-7).  The full experiment (256 x 64, 2000 training seeds to r <= 1e-6,
200 held-out seeds to r <= 1e-8 with residual checks every 1000 steps) runs with
LBM_WARMSTART_FULL=1; it prints one JSON line with every measurement.  In that mode
LBM_WARMSTART_TRAIN / _TEST set the seed counts, _TRAIN_TOL / _TRAIN_MAX how far the
training channels are run, _TOL the held-out tolerance, _PLAIN how many held-out channels
are also timed one by one, and LBM_WARMSTART_VARIANTS=0 drops the surrogate's partial
starts (temperature alone; temperature, interface and velocity)."""
import json
import os

import numpy as np
import pytest

import lbm_workloads as WL

pytestmark = pytest.mark.gpu


def closed_form_T(c):
    from oracle import analytic as A
    d, p = c["domain"], c["params"]
    ch = A.Channel(l=d["nx"] / max(d["heat_periods"], 1), a=d["ny"] - d["b"], b=d["b"], k_ratio=p["cond_ratio"],
                   mu_ratio=p["visc_ratio"], mu_b=(p["tau_flow"] - 0.5) / 3.0, sigma_T=p["sigma1"],
                   sigma_TT=p["sigma2"], T_h=p["T_hot"], T_c=p["T_cold"], T_ref=p["T_ref"], dT=p["dT"])
    x = np.arange(d["nx"])[None, :] * np.ones((d["ny"], 1))
    y = (np.arange(d["ny"])[:, None] + 0.5 - d["b"]) * np.ones((1, d["nx"]))
    return A.temperature(ch, x, y)


def run(full: bool):
    import paper_2210_07501_gb300 as pkg
    from paper_2210_07501_gb300 import warmstart
    pkg.build()
    pkg.load()
    if full:
        train = WL.surrogate_cases(int(os.environ.get("LBM_WARMSTART_TRAIN", "2000")), seed=1000)
        test = WL.surrogate_cases(int(os.environ.get("LBM_WARMSTART_TEST", "200")), seed=2000)
        env = os.environ.get
        kw = dict(tol=float(env("LBM_WARMSTART_TOL", "1e-8")), max_steps=3000000, K=1000,
                  train_tol=float(env("LBM_WARMSTART_TRAIN_TOL", "1e-6")),
                  train_max_steps=int(env("LBM_WARMSTART_TRAIN_MAX", "400000")), iters=3000, batch=16, lr=1e-3,
                  plain_cases=int(env("LBM_WARMSTART_PLAIN", "0")), variants=env("LBM_WARMSTART_VARIANTS", "1") == "1")
    else:
        train = WL.surrogate_cases(96, seed=11, nx=64, ny=32)
        test = WL.surrogate_cases(8, seed=12, nx=64, ny=32)
        kw = dict(tol=1e-7, max_steps=300000, K=100, train_tol=1e-6, train_max_steps=150000, iters=1500, batch=16,
                  lr=2e-3)
    extra = {"closed_form_T": [{"T": closed_form_T(c)} for c in test]}
    return warmstart.experiment(train, test, extra_starts=extra,
                                progress=lambda name, d: print(json.dumps({"phase": name, **d}), flush=True), **kw)


def test_warm_start_against_cold_and_closed_form():
    pytest.importorskip("torch")
    full = os.environ.get("LBM_WARMSTART_FULL") == "1"
    r = run(full)
    print(json.dumps(r))
    cf = r["variants"]["closed_form_T"]
    v = r["variants"]
    print(f"mean steps to r <= {r['tol']:g}: cold {r['cold_steps_mean']:.0f}, closed-form T "
          f"{cf['steps_mean']:.0f}, surrogate T + phi {r['warm_steps_mean']:.0f}" +
          "".join(f", {k} {v[k]['steps_mean']:.0f}" for k in ("surrogate_T", "surrogate_T_phi_u_v") if k in v))
    if full:
        # 256 x 64 to r <= 1e-8: the settling of the interface, which the conservative phase
        # field does by redistributing phi along the channel (a time of order L^2 / M_phi ~
        # 6.5e5 steps), sets the step count for every start, and the surrogate trained on
        # channels stopped at r <= 1e-6 predicts that settled interface poorly (measured
        # means: ~1.95M steps for every start, 136 of 200 held-out channels converged within
        # 3M steps); the measurements are printed, not asserted
        assert r["cold_converged"] >= 0.5 * r["test_cases"]
        return
    assert r["loss_last"] < 0.05 * r["loss_first"]
    assert r["cold_converged"] == r["test_cases"] and r["warm_converged"] == r["test_cases"]
    # the surrogate start (temperature and interface) gains over the plain cold start and
    # over the closed-form temperature, which leaves the slow settling of the interface
    # (measured on the default case: 99,962 mean steps against 147,625 cold and 147,538
    # from the closed-form temperature)
    assert r["warm_steps_mean"] < 0.9 * r["cold_steps_mean"]
    assert r["warm_steps_mean"] < 0.9 * cf["steps_mean"]
    assert r["warm_fewer_steps_cases"] >= 0.75 * r["test_cases"]
    # the surrogate's temperature against the converged LB one (the reference); measured
    # 0.10 on the default case (96 training channels, 1500 iterations)
    assert r["surrogate_rel_l2_vs_lb"]["T"] < 0.2
    # warm- and cold-started runs converge to the same LB solution
    assert r["warm_vs_cold_final_rel_l2"]["T"] < 1e-3
    assert r["warm_vs_cold_final_rel_l2"]["phi"] < 1e-3
