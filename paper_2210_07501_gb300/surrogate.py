"""Inputs and targets of the warm-start surrogate (host-side preparation).

The surrogate maps a channel's parameters, heating profile and geometry to its steady
fields.  It sees nothing of the method's solution: its inputs are

  [12][ny][nx]: cos(2 pi k x / nx) and sin(2 pi k x / nx) (the bottom-wall heating
  profile), y / ny, the bottom-layer mask (y < b), (y - b) / ny, the initial interface
  profile phi_flat(y) = 1/2 + 1/2 tanh(2 (y - b) / W) (what lbm_init_fields builds), the
  heating profile faded linearly to the isothermal top wall, cos(2 pi k x / nx) (1 - y / ny),
  and five constant channels with the scaled parameters sigma1, sigma2, a / b, the
  conductivity ratio and the viscosity ratio;

and its targets [4][ny][nx] are the LB steady state itself:

  (phi - phi_flat) / PHI_SCALE   the steady interface's departure from the flat profile,
  T - T_ref,
  u / U, v / U                    with U = (|sigma1| + 2 |sigma2| dT) dT (b / l) / mu_b, the
                                  order of magnitude of a Marangoni velocity: the surface
                                  tension difference along the interface over a viscous
                                  stress (a scale, used only to bring u, v to O(1)).
"""
from __future__ import annotations

import numpy as np

N_IN = 12
PARAM_SCALE = {"sigma1": 2e-5, "sigma2": 4e-4, "ab": 4.0, "cond_ratio": 4.0, "visc_ratio": 4.0}
PHI_SCALE = 1e-3


def velocity_scale(domain: dict, params: dict) -> float:
    b = float(domain["b"])
    l = float(domain["nx"]) / max(int(domain["heat_periods"]), 1)
    mu_b = params.get("rho_bottom", 1.0) * (params["tau_flow"] - 0.5) / 3.0
    dT = abs(params["dT"])
    return max((abs(params["sigma1"]) + 2.0 * abs(params["sigma2"]) * dT) * dT * (b / l) / mu_b, 1e-12)


def _grid(domain: dict):
    nx, ny = int(domain["nx"]), int(domain["ny"])
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    y = (np.arange(ny)[:, None] + 0.5) * np.ones((1, nx))
    return x, y


def phi_flat(domain: dict) -> np.ndarray:
    """The flat tanh interface of width W at y = b on the nodes (the default initial phi)."""
    _, y = _grid(domain)
    return 0.5 + 0.5 * np.tanh(2.0 * (y - float(domain["b"])) / float(domain["W"]))


def features(domain: dict, params: dict) -> np.ndarray:
    nx, ny, k = int(domain["nx"]), int(domain["ny"]), max(int(domain["heat_periods"]), 1)
    b = float(domain["b"])
    x, y = _grid(domain)
    c = np.cos(2 * np.pi * k * x / nx)
    ch = [c, np.sin(2 * np.pi * k * x / nx), y / ny, (y < b).astype(float), (y - b) / ny, phi_flat(domain),
          c * (1.0 - y / ny)]
    ab = (ny - b) / b
    for key, val in (("sigma1", params["sigma1"]), ("sigma2", params["sigma2"]), ("ab", ab),
                     ("cond_ratio", params["cond_ratio"]), ("visc_ratio", params["visc_ratio"])):
        ch.append(np.full((ny, nx), val / PARAM_SCALE[key]))
    out = np.stack(ch).astype(np.float32)
    assert out.shape[0] == N_IN
    return out


def targets(domain: dict, params: dict, fields: dict) -> np.ndarray:
    U = velocity_scale(domain, params)
    return np.stack([(fields["phi"] - phi_flat(domain)) / PHI_SCALE, fields["T"] - params["T_ref"],
                     fields["u"] / U, fields["v"] / U]).astype(np.float32)


def fields_from_prediction(domain: dict, params: dict, pred: np.ndarray, use_phi: bool = False,
                           use_velocity: bool = False) -> dict:
    """Predicted [4][ny][nx] (target units) back to initial fields for lbm_init_fields
    (pressure left at p0).

    T always.  With use_phi, phi = phi_flat + the predicted departure, made mass-neutral:
    the Allen-Cahn lattice conserves sum phi, so a prediction that adds or removes phi
    would move the steady interface for good; the net amount is taken out as a uniform
    shift of the flat profile (along d phi_flat / dy).  With use_velocity, u and v too."""
    U = velocity_scale(domain, params)
    out = {"T": params["T_ref"] + pred[1].astype(np.float64)}
    if use_phi:
        base = phi_flat(domain)
        d = PHI_SCALE * pred[0].astype(np.float64)
        w = 1.0 - (2.0 * base - 1.0) ** 2          # proportional to d phi_flat / dy
        d -= w * (d.sum() / w.sum())
        out["phi"] = np.clip(base + d, 0.0, 1.0)
    if use_velocity:
        out["u"] = U * pred[2].astype(np.float64)
        out["v"] = U * pred[3].astype(np.float64)
    return out
