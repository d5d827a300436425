"""Peak interfacial velocity U_max against the property ratios and the surface-tension
coefficients (the paper's parametric study of Sec. 6: U_max versus k~, mu~, M1 and M2 for
a/b = 1/3, 1 and 3), computed as one batched sweep to steady state.

Base case (Sec. 6): a 200 x 100 channel, l = 200, a + b = 100, T_h = T_c = T_ref = dT = 1,
sigma0 = 1e-3, M1 = sigma_T dT / sigma0 = 0, M2 = sigma_TT dT^2 / sigma0 = 5e-2, D2Q9 for all
three lattices, W = 5, M_phi = 0.02.  The relaxation times are not printed for this study:
tau_flow = tau_T = 1.5 (nu_b = alpha_b = 1/3).  The steady creeping-flow state depends on the
viscosity and conductivity ratios and on mu_b, not on the diffusivities, and the larger nu_b
and alpha_b shorten the approach to it and keep tau moderate at the ratios 1/4 and 4.
At these coefficients the interface velocity is ~1e-7: FP64 storage (FP32 storage resolves
velocities down to ~1e-8 of the populations only).

U_max is the largest |u| on the interface, taken as the mean of the two node rows that
straddle it (y = b -/+ 1/2).  Every step of the sweep runs in the CUDA library; comparisons
with the closed-form solution of Sec. 3 are made by the callers that hold one.
"""
from __future__ import annotations

import numpy as np

from .warmstart import steady_batch

AB = (1.0 / 3.0, 1.0, 3.0)


def base(ab: float, **over) -> dict:
    ny, nx = 100, 200
    b = float(round(ny / (1.0 + ab)))
    p = dict(sigma0=1e-3, sigma1=0.0, sigma2=5e-2 * 1e-3, T_ref=1.0, T_hot=1.0, T_cold=1.0, dT=1.0,
             tau_flow=1.5, visc_ratio=1.0, tau_T=1.5, cond_ratio=1.0, tau_phi=0.56,
             rho_bottom=1.0, rho_top=1.0, Fx_ext=0.0, Fy_ext=0.0)
    for k, v in over.items():
        if k == "M1":
            p["sigma1"] = v * p["sigma0"] / p["dT"]
        elif k == "M2":
            p["sigma2"] = v * p["sigma0"] / p["dT"] ** 2
        elif k == "visc_ratio":
            # the top viscosity stays at its base value and the bottom one is mu_a / mu~: the
            # reading under which U_max rises with mu~ as Sec. 6 describes (with mu_b held
            # fixed instead, the closed form falls with mu~)
            p["visc_ratio"] = v
            p["tau_flow"] = 3.0 * ((p["tau_flow"] - 0.5) / 3.0) / v + 0.5
        else:
            p[k] = v
    label = f"ab={ab:.3g}," + ",".join(f"{k}={v:g}" for k, v in over.items())
    return {"name": "trend-" + label, "domain": dict(nx=nx, ny=ny, b=b, W=5.0, heat_periods=1, q_phi=9, q_T=9),
            "params": p}


def cases(param: str, values, ab_values=AB) -> list:
    """One case per (a/b, value); param is 'cond_ratio', 'visc_ratio', 'M1' or 'M2'."""
    return [base(ab, **{param: v}) for ab in ab_values for v in values]


def interface_u_max(u: np.ndarray, b: float) -> float:
    j = int(round(b))
    return float(np.max(np.abs(0.5 * (u[j - 1] + u[j]))))


def run(case_list: list, precision: str = "fp64", tol: float = 1e-6, max_steps: int = 200000, stream=None):
    fields, steps, conv, seconds = steady_batch(case_list, tol, max_steps, precision, stream=stream)
    out = []
    for c, f, n, ok in zip(case_list, fields, steps, conv):
        out.append({"name": c["name"], "b": c["domain"]["b"], "params": c["params"], "steps": int(n),
                    "converged": bool(ok), "U_lb": interface_u_max(f["u"], c["domain"]["b"])})
    return out, seconds


# ---- interface deformation at larger capillary numbers (Sec. 6, last study) ----
# a/b = 3 in the 200 x 100 channel (b = 25), M1 = 0, sigma0 = 1e-3, k~ = mu~ = 1; the paper
# raises M2 to 3, 5, 10, 20 (Ca = 0.34 .. 2.29) and shows the interface deforming more with
# Ca while the eight cells persist.  Relaxation times as the Sec. 6 SRF channel (tau_flow =
# 1.17, tau_T = 2.73, tau_phi = 0.56); velocities reach ~1e-2, so FP32 storage suffices.

def deformation_case(M2: float) -> dict:
    p = dict(sigma0=1e-3, sigma1=0.0, sigma2=M2 * 1e-3, T_ref=1.0, T_hot=1.0, T_cold=1.0, dT=1.0,
             tau_flow=1.17, visc_ratio=1.0, tau_T=2.73, cond_ratio=1.0, tau_phi=0.56,
             rho_bottom=1.0, rho_top=1.0, Fx_ext=0.0, Fy_ext=0.0)
    return {"name": f"deformation-M2={M2:g}", "domain": dict(nx=200, ny=100, b=25.0, W=5.0, heat_periods=1,
                                                             q_phi=9, q_T=9), "params": p}


def interface_height(phi: np.ndarray) -> np.ndarray:
    """Per column, the height where phi crosses 1/2 (linear between nodes at y = j + 1/2),
    searched upwards from the bottom wall."""
    ny, nx = phi.shape
    h = np.full(nx, np.nan)
    for i in range(nx):
        col = phi[:, i] - 0.5
        j = np.flatnonzero((col[:-1] < 0) & (col[1:] >= 0))
        if j.size:
            j = j[0]
            h[i] = j + 0.5 + col[j] / (col[j] - col[j + 1])
    return h


def cell_count(v: np.ndarray, b: float) -> int:
    """Convection cells: sign changes of v along x at mid-height of each layer, summed."""
    ny = v.shape[0]
    total = 0
    for y in (0.5 * b, b + 0.5 * (ny - b)):
        row = v[int(y)]
        s = np.sign(np.where(np.abs(row) <= 1e-12 * max(np.abs(row).max(), 1e-300), 0.0, row))
        s = s[s != 0]
        total += int(np.sum(s != np.roll(s, 1))) if s.size else 0
    return total


def run_deformation(M2_values=(0.1, 3.0, 5.0, 10.0, 20.0), precision: str = "fp32", tol: float = 1e-5,
                    max_steps: int = 150000, stream=None):
    cl = [deformation_case(m) for m in M2_values]
    fields, steps, conv, seconds = steady_batch(cl, tol, max_steps, precision, stream=stream)
    out = []
    for c, f, n, ok in zip(cl, fields, steps, conv):
        h = interface_height(f["phi"])
        out.append({"name": c["name"], "M2": c["params"]["sigma2"] / c["params"]["sigma0"], "steps": int(n),
                    "converged": bool(ok), "deflection": float(np.nanmax(h) - np.nanmin(h)),
                    "mean_height": float(np.nanmean(h)), "cells": cell_count(f["v"], c["domain"]["b"]),
                    "u_max": float(np.abs(f["u"]).max()), "height": h})
    return out, seconds


# ---- steady state of the 1024 x 256 channel ----
# a = b = 128, W = 5, sigma2 = -2e-4, sigma1 in {0, 2e-5}, mu~ = k~ = 2, tau_b = 0.8.  The run
# starts from the caller's initial fields (e.g. a temperature close to the steady one: the
# slowest mode of the approach to steady state from rest is thermal) and stops at r <= tol
# or max_steps; it returns the steady fields and the interface velocity.

def steady(cases: list, init=None, precision: str = "fp64", tol: float = 1e-8, max_steps: int = 1500000,
           stream=None) -> list:
    fields, steps, conv, seconds = steady_batch(cases, tol, max_steps, precision, init=init, stream=stream)
    return [{"name": c["name"], "steps": int(n), "converged": bool(ok), "seconds": seconds,
             "U_lb": interface_u_max(f["u"], c["domain"]["b"]), "fields": f}
            for c, f, n, ok in zip(cases, fields, steps, conv)]
