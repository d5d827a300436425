"""Inputs and targets of the warm-start surrogate (host-side preparation).

Input channels [9][ny][nx] of one channel case: cos(2 pi k x / nx) (the heating profile),
sin(2 pi k x / nx), y / ny, the layer mask (1 in the bottom layer y < b), and five constant
channels with the scaled parameters sigma1, sigma2, a/b, conductivity ratio, viscosity ratio.

Targets [4][ny][nx]: phi, T - T_ref, u / U and v / U, with the velocity scale
U = (|sigma1| + 2 |sigma2| dT) dT (b / l) / mu_b from the Marangoni stress balance of
App. C (the magnitude, not the sign), so that every case has O(1) targets.
"""
from __future__ import annotations

import numpy as np

PARAM_SCALE = {"sigma1": 2e-5, "sigma2": 4e-4, "ab": 4.0, "cond_ratio": 4.0, "visc_ratio": 4.0}


def velocity_scale(domain: dict, params: dict) -> float:
    b = float(domain["b"])
    l = float(domain["nx"]) / max(int(domain["heat_periods"]), 1)
    mu_b = params.get("rho_bottom", 1.0) * (params["tau_flow"] - 0.5) / 3.0
    dT = abs(params["dT"])
    return max((abs(params["sigma1"]) + 2.0 * abs(params["sigma2"]) * dT) * dT * (b / l) / mu_b, 1e-12)


def features(domain: dict, params: dict) -> np.ndarray:
    nx, ny, k = int(domain["nx"]), int(domain["ny"]), max(int(domain["heat_periods"]), 1)
    b = float(domain["b"])
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    y = (np.arange(ny)[:, None] + 0.5) * np.ones((1, nx))
    ab = (ny - b) / b
    ch = [np.cos(2 * np.pi * k * x / nx), np.sin(2 * np.pi * k * x / nx), y / ny, (y < b).astype(float)]
    for key, val in (("sigma1", params["sigma1"]), ("sigma2", params["sigma2"]), ("ab", ab),
                     ("cond_ratio", params["cond_ratio"]), ("visc_ratio", params["visc_ratio"])):
        ch.append(np.full((ny, nx), val / PARAM_SCALE[key]))
    return np.stack(ch).astype(np.float32)


def targets(domain: dict, params: dict, fields: dict) -> np.ndarray:
    U = velocity_scale(domain, params)
    return np.stack([fields["phi"], fields["T"] - params["T_ref"], fields["u"] / U, fields["v"] / U]).astype(np.float32)


def fields_from_prediction(domain: dict, params: dict, pred: np.ndarray, use_phi: bool = False) -> dict:
    """Predicted [4][ny][nx] back to initial fields for lbm_init_fields (pressure left at p0).

    The predicted phi is left out by default: phi is conserved by the Allen-Cahn lattice, so
    any error in the predicted sum of phi has to be undone by slow interface diffusion, while
    at the small capillary numbers of these channels the steady phi is the tanh profile at the
    given interface height, which lbm_init_fields builds when phi is omitted."""
    U = velocity_scale(domain, params)
    out = {"T": params["T_ref"] + pred[1].astype(np.float64), "u": U * pred[2].astype(np.float64),
           "v": U * pred[3].astype(np.float64)}
    if use_phi:
        out["phi"] = np.clip(pred[0].astype(np.float64), 0.0, 1.0)
    return out
