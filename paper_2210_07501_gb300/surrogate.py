"""Inputs and targets of the warm-start surrogate (host-side preparation).

Input channels [12][ny][nx] of one channel case: cos(2 pi k x / nx) (the heating profile),
sin(2 pi k x / nx), y / ny, the layer mask (1 in the bottom layer y < b), five constant
channels with the scaled parameters sigma1, sigma2, a/b, conductivity ratio, viscosity
ratio, and the sharp-interface creeping-flow solution of Sec. 3 (T - T_ref, u / U, v / U),
so that the network learns the correction of the diffuse-interface LB steady state to it.

Targets [4][ny][nx]: phi and the corrections of the LB steady state to the closed form,
T - T_cf, (u - u_cf) / U and (v - v_cf) / U, with the velocity scale
U = (|sigma1| + 2 |sigma2| dT) dT (b / l) / mu_b from the Marangoni stress balance of
App. C (the magnitude, not the sign).  The network's last layer starts near zero, so an
untrained network already reproduces the closed form and training learns the diffuse-
interface correction.
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


def closed_form(domain: dict, params: dict):
    """T, u, v of the two-layer creeping-flow solution (Sec. 3.1, 3.2; App. A) on the lattice
    nodes: x from the heating peak, y from the interface (y = j + 1/2 - b), a = ny - b on top,
    b below; u = d(psi)/dy, v = -d(psi)/dx."""
    nx, ny, k = int(domain["nx"]), int(domain["ny"]), max(int(domain["heat_periods"]), 1)
    b = float(domain["b"])
    a = ny - b
    l = nx / k
    w = 2 * np.pi / l
    at, bt = a * w, b * w
    kr, mr = params["cond_ratio"], params["visc_ratio"]
    mu_b = params.get("rho_bottom", 1.0) * (params["tau_flow"] - 0.5) / 3.0
    Th, Tc, Tr, dT = params["T_hot"], params["T_cold"], params["T_ref"], params["dT"]
    sT, sTT = params["sigma1"], params["sigma2"]
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    y = (np.arange(ny)[:, None] + 0.5 - b) * np.ones((1, nx))
    f = 1.0 / (kr * np.sinh(bt) * np.cosh(at) + np.sinh(at) * np.cosh(bt))
    den = a + b * kr
    Ta = ((Tc - Th) * y + Tc * kr * b + Th * a) / den + dT * f * np.sinh(at - w * y) * np.cos(w * x)
    Tb = (kr * (Tc - Th) * y + Tc * kr * b + Th * a) / den + \
        dT * f * (np.sinh(at) * np.cosh(w * y) - kr * np.sinh(w * y) * np.cosh(at)) * np.cos(w * x)
    T = np.where(y >= 0, Ta, Tb)

    def hfun(p, q):
        Sp, Sq = np.sinh(p) ** 2 - p ** 2, np.sinh(q) ** 2 - q ** 2
        return Sp * Sq / (mr * Sq * (np.sinh(2 * p) - 2 * p) + Sp * (np.sinh(2 * q) - 2 * q))

    g = np.sinh(at) * f
    Tm = (Tc * kr * b + Th * a) / den
    Ut = -(dT / mu_b) * g * hfun(at, bt) * (sT + 2 * sTT * (Tm - Tr))
    Utt = -(sTT * dT ** 2 / mu_b) * g ** 2 * hfun(2 * at, 2 * bt)

    def consts(t, L, sign, m):
        S_ = np.sinh(m * t) ** 2 - (m * t) ** 2
        return (np.sinh(m * t) ** 2 / S_, -m * L * t / S_, sign * (np.sinh(2 * m * t) - 2 * m * t) / (2 * S_))

    u = np.zeros_like(y)
    v = np.zeros_like(y)
    for top, L, sign in ((True, a, -1.0), (False, b, 1.0)):
        C2, C3, C4 = consts(at if top else bt, L, sign, 1)
        D2, D3, D4 = consts(at if top else bt, L, sign, 2)
        uu = Ut * ((C2 + w * (C3 + C4 * y)) * np.cosh(w * y) + (C4 + w * C2 * y) * np.sinh(w * y)) * np.sin(w * x) \
            + 0.5 * Utt * ((D2 + 2 * w * (D3 + D4 * y)) * np.cosh(2 * w * y)
                           + (D4 + 2 * w * D2 * y) * np.sinh(2 * w * y)) * np.sin(2 * w * x)
        vv = -w * Ut * (C2 * y * np.cosh(w * y) + (C3 + C4 * y) * np.sinh(w * y)) * np.cos(w * x) \
            - w * Utt * (D2 * y * np.cosh(2 * w * y) + (D3 + D4 * y) * np.sinh(2 * w * y)) * np.cos(2 * w * x)
        sel = (y >= 0) if top else (y < 0)
        u = np.where(sel, uu, u)
        v = np.where(sel, vv, v)
    return T, u, v


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
    T, u, v = closed_form(domain, params)
    U = velocity_scale(domain, params)
    ch += [T - params["T_ref"], u / U, v / U]
    return np.stack(ch).astype(np.float32)


def closed_form_fields(domain: dict, params: dict) -> dict:
    """The closed-form T, u, v as initial fields (phi from lbm_init_fields' tanh profile)."""
    T, u, v = closed_form(domain, params)
    return {"T": T, "u": u, "v": v}


def targets(domain: dict, params: dict, fields: dict) -> np.ndarray:
    U = velocity_scale(domain, params)
    T, u, v = closed_form(domain, params)
    return np.stack([fields["phi"], fields["T"] - T, (fields["u"] - u) / U, (fields["v"] - v) / U]).astype(np.float32)


def fields_from_prediction(domain: dict, params: dict, pred: np.ndarray, use_phi: bool = False,
                           use_velocity: bool = True) -> dict:
    """Predicted [4][ny][nx] back to initial fields for lbm_init_fields (pressure left at p0).

    The predicted phi is left out by default: phi is conserved by the Allen-Cahn lattice, so
    any error in the predicted sum of phi has to be undone by slow interface diffusion, while
    at the small capillary numbers of these channels the steady phi is the tanh profile at the
    given interface height, which lbm_init_fields builds when phi is omitted."""
    U = velocity_scale(domain, params)
    T, u, v = closed_form(domain, params)
    out = {"T": T + pred[1].astype(np.float64)}
    if use_velocity:
        out["u"] = u + U * pred[2].astype(np.float64)
        out["v"] = v + U * pred[3].astype(np.float64)
    if use_phi:
        out["phi"] = np.clip(pred[0].astype(np.float64), 0.0, 1.0)
    return out
