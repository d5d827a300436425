"""The paper's droplet workloads on the GPU path.

* Thermocapillary migration of a 2-D drop (Sec. 5.1): the drop of radius R in a uniform
  temperature gradient moves towards lower surface tension; its velocity, from the
  centroid of phi, is compared with the Young-Goldstein-Block terminal velocity
  U_YGB = 2 U* / ((2 + k~)(2 + 3 mu~)), U* = |sigma_T| |grad T| R / mu (the 3-D creeping
  flow result; 2-D drops settle near 0.8 U_YGB).
* Static drop (Laplace's law): with constant sigma the pressure jump across a drop of
  radius R is sigma / R in 2-D.

Every step runs in the CUDA library; this module only sets up fields and reads them.
"""
from __future__ import annotations

import time

import numpy as np

from . import Lbm


def u_ygb(sigma_T: float, grad_T: float, R: float, mu: float, k_ratio: float = 1.0, mu_ratio: float = 1.0):
    """Young-Goldstein-Block terminal velocity (Sec. 5.1)."""
    u_star = abs(sigma_T) * abs(grad_T) * R / mu
    return 2.0 * u_star / ((2.0 + k_ratio) * (2.0 + 3.0 * mu_ratio))


def centroid(phi: np.ndarray):
    """Centroid (x, y) of phi; node (i, j) sits at (i, j + 1/2)."""
    ny, nx = phi.shape
    m = phi.sum()
    return float((phi.sum(axis=0) * np.arange(nx)).sum() / m), float((phi.sum(axis=1) * (np.arange(ny) + 0.5)).sum() / m)


def migration(w: dict, R: float, t_star_end: float = 2.5, samples: int = 50, precision: str = "fp64",
              stream=None) -> dict:
    """Run the drop case `w` (walls at T_hot below, T_cold above) from rest until
    t* = t U_YGB / R reaches t_star_end; returns the centroid track, the velocity between
    samples, U_YGB and the wall time."""
    import lbm_workloads as WL
    d, p = w["domain"], w["params"]
    nx, ny = d["nx"], d["ny"]
    grad_T = (p["T_cold"] - p["T_hot"]) / ny
    mu = (p["tau_flow"] - 0.5) / 3.0 * p["rho_bottom"]
    uy = u_ygb(p["sigma1"], grad_T, R, mu, p["cond_ratio"], p["visc_ratio"])
    steps_total = int(round(t_star_end * R / uy))
    every = max(1, steps_total // samples)
    g = Lbm(d, p, precision=precision, stream=stream)
    g.lbm_set_check_interval(1 << 30)   # no residual checks
    g.lbm_init_fields(**WL.drop_fields(nx, ny, R, d["W"], p["T_hot"], p["T_cold"]))
    t, yc, xc = [0], [], []
    f = g.lbm_fields()
    cx, cy = centroid(f["phi"])
    xc.append(cx), yc.append(cy)
    t0 = time.perf_counter()
    done = 0
    while done < steps_total:
        n = min(every, steps_total - done)
        g.lbm_step(n)
        done += n
        f = g.lbm_fields()
        cx, cy = centroid(f["phi"])
        t.append(done), xc.append(cx), yc.append(cy)
    wall = time.perf_counter() - t0
    mass = g.lbm_diag()["mass"]
    g.close()
    t = np.asarray(t, float)
    yc = np.asarray(yc)
    vel = np.diff(yc) / np.diff(t)
    return {"t": t, "t_star": t * uy / R, "x_c": np.asarray(xc), "y_c": yc, "U": vel, "U_ygb": uy,
            "U_over_U_ygb": vel / uy, "steps": steps_total, "seconds": wall, "mass": mass,
            "nodes": nx * ny, "precision": precision}


def laplace(n: int, R: float, sigma: float, W: float = 4.0, steps: int = 6000, precision: str = "fp64",
            tau_flow: float = 1.0, stream=None) -> dict:
    """Static drop of radius R at the centre of an n x n box (periodic x, walls in y) with
    constant sigma: the pressure jump between the centre and a corner region."""
    import lbm_workloads as WL
    w = WL.channel(n, n, n / 2, W=W, sigma0=sigma, sigma1=0.0, sigma2=0.0, dT=0.0, tau_flow=tau_flow)
    d, p = w["domain"], w["params"]
    g = Lbm(d, p, precision=precision, stream=stream)
    g.lbm_set_check_interval(1 << 30)   # no residual checks
    g.lbm_init_fields(**WL.drop_fields(n, n, R, W, p["T_hot"], p["T_cold"]))
    g.lbm_step(steps)
    f = g.lbm_fields()
    g.close()
    dp = f["dp"]
    c = n // 2
    inside = dp[c - 2:c + 2, c - 2:c + 2].mean()
    outside = dp[1:5, 1:5].mean()
    return {"R": R, "jump": float(inside - outside), "sigma_over_R": sigma / R,
            "ratio": float((inside - outside) * R / sigma), "u_max": float(np.abs(f["u"]).max())}
