"""Closed-form creeping-flow solution for two superimposed layers (arXiv 2210.07501).

TEST INFRASTRUCTURE ONLY (part of the oracle): pins the LB oracle against the paper's
analysis.  Coordinates follow the paper: x from the heating peak, y from the interface,
fluid 'a' on top (0 <= y <= a), fluid 'b' at the bottom (-b <= y <= 0), omega = 2 pi / l.

Sources:
  temperature     Sec. 3.1 and App. A (f(a~, b~, k~), Q^a, Q^b, P^a, P^b)
  stream function Sec. 3.2 (constants C_j, D_j; U_t, U_tt, g, h, h~1)
  velocities      Sec. 3.2, read with u = +d(psi)/dy, v = -d(psi)/dx, which is what
                  the printed velocity formulas differentiate to (the printed definition
                  u = -d(psi)/dy is not divergence-free together with v = -d(psi)/dx)
  velocity scale  App. C (U_s); droplet migration speed Sec. 5.1 (U_YGB).
Parity: pinned by tests/test_analytic.py (wall no-slip, interface stress balance,
continuity, Laplace/biharmonic residuals, and the numbers the paper prints).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Channel:
    l: float            # period length along x
    a: float            # top-layer thickness
    b: float            # bottom-layer thickness
    k_ratio: float      # k_a / k_b
    mu_ratio: float     # mu_a / mu_b
    mu_b: float         # bottom dynamic viscosity
    sigma_T: float
    sigma_TT: float
    T_h: float = 1.0
    T_c: float = 1.0
    T_ref: float = 1.0
    dT: float = 1.0

    @property
    def omega(self):
        return 2.0 * np.pi / self.l

    @property
    def at(self):
        return self.a * self.omega

    @property
    def bt(self):
        return self.b * self.omega


def f_fun(at, bt, k):
    """App. A: f(a~, b~, k~)."""
    return 1.0 / (k * np.sinh(bt) * np.cosh(at) + np.sinh(at) * np.cosh(bt))


def h_fun(at, bt, mu):
    """Sec. 3.2: h(a~, b~, mu~)."""
    Sa = np.sinh(at) ** 2 - at ** 2
    Sb = np.sinh(bt) ** 2 - bt ** 2
    return Sa * Sb / (mu * Sb * (np.sinh(2 * at) - 2 * at) + Sa * (np.sinh(2 * bt) - 2 * bt))


def temperature(c: Channel, x, y):
    """T^a for y >= 0 and T^b for y < 0 (Sec. 3.1)."""
    x = np.asarray(x, dtype=float)
    y = np.asarray(y, dtype=float)
    w, at, k = c.omega, c.at, c.k_ratio
    f = f_fun(at, c.bt, k)
    den = c.a + c.b * k
    Ta = ((c.T_c - c.T_h) * y + c.T_c * k * c.b + c.T_h * c.a) / den \
        + c.dT * f * np.sinh(at - w * y) * np.cos(w * x)
    Tb = (k * (c.T_c - c.T_h) * y + c.T_c * k * c.b + c.T_h * c.a) / den \
        + c.dT * f * (np.sinh(at) * np.cosh(w * y) - k * np.sinh(w * y) * np.cosh(at)) * np.cos(w * x)
    return np.where(y >= 0.0, Ta, Tb)


def U_t(c: Channel):
    """Sec. 3.2: amplitude of the first harmonic of the interface velocity."""
    g = np.sinh(c.at) * f_fun(c.at, c.bt, c.k_ratio)
    h = h_fun(c.at, c.bt, c.mu_ratio)
    Tm = (c.T_c * c.k_ratio * c.b + c.T_h * c.a) / (c.a + c.b * c.k_ratio)
    return -(c.dT / c.mu_b) * g * h * (c.sigma_T + 2.0 * c.sigma_TT * (Tm - c.T_ref))


def U_tt(c: Channel):
    """Sec. 3.2: amplitude (times 2) of the second harmonic; h~1 = h(2a~, 2b~, mu~)."""
    g = np.sinh(c.at) * f_fun(c.at, c.bt, c.k_ratio)
    return -(c.sigma_TT * c.dT ** 2 / c.mu_b) * g ** 2 * h_fun(2 * c.at, 2 * c.bt, c.mu_ratio)


def constants(c: Channel):
    """Sec. 3.2: C_j^{a,b} (first harmonic) and D_j^{a,b} (second harmonic), j = 1..4."""
    at, bt, a, b = c.at, c.bt, c.a, c.b

    def set_(t, L, sign):
        S = np.sinh(t) ** 2 - t ** 2
        return (0.0, np.sinh(t) ** 2 / S, -L * t / S, sign * (np.sinh(2 * t) - 2 * t) / (2 * S))

    def set2(t, L, sign):
        S = np.sinh(2 * t) ** 2 - 4 * t ** 2
        return (0.0, np.sinh(2 * t) ** 2 / S, -2 * L * t / S, sign * (np.sinh(4 * t) - 4 * t) / (2 * S))

    return {"Ca": set_(at, a, -1.0), "Cb": set_(bt, b, +1.0),
            "Da": set2(at, a, -1.0), "Db": set2(bt, b, +1.0)}


def velocity(c: Channel, x, y):
    """(u, v) from the printed velocity formulas of Sec. 3.2 (a for y >= 0, b below)."""
    x = np.asarray(x, dtype=float)
    y = np.asarray(y, dtype=float)
    w = c.omega
    Ut, Utt = U_t(c), U_tt(c)
    K = constants(c)

    def uv(C, D):
        _, C2, C3, C4 = C
        _, D2, D3, D4 = D
        u = Ut * ((C2 + w * (C3 + C4 * y)) * np.cosh(w * y) + (C4 + w * C2 * y) * np.sinh(w * y)) * np.sin(w * x) \
            + 0.5 * Utt * ((D2 + 2 * w * (D3 + D4 * y)) * np.cosh(2 * w * y)
                           + (D4 + 2 * w * D2 * y) * np.sinh(2 * w * y)) * np.sin(2 * w * x)
        v = -w * Ut * (C2 * y * np.cosh(w * y) + (C3 + C4 * y) * np.sinh(w * y)) * np.cos(w * x) \
            - w * Utt * (D2 * y * np.cosh(2 * w * y) + (D3 + D4 * y) * np.sinh(2 * w * y)) * np.cos(2 * w * x)
        return u, v

    ua, va = uv(K["Ca"], K["Da"])
    ub, vb = uv(K["Cb"], K["Db"])
    top = y >= 0.0
    return np.where(top, ua, ub), np.where(top, va, vb)


def stream_function(c: Channel, x, y):
    """psi with u = d(psi)/dy, v = -d(psi)/dx, from the constants of Sec. 3.2."""
    x = np.asarray(x, dtype=float)
    y = np.asarray(y, dtype=float)
    w = c.omega
    Ut, Utt = U_t(c), U_tt(c)
    K = constants(c)

    def ps(C, D):
        _, C2, C3, C4 = C
        _, D2, D3, D4 = D
        return Ut * (C2 * y * np.cosh(w * y) + (C3 + C4 * y) * np.sinh(w * y)) * np.sin(w * x) \
            + 0.5 * Utt * (D2 * y * np.cosh(2 * w * y) + (D3 + D4 * y) * np.sinh(2 * w * y)) * np.sin(2 * w * x)

    return np.where(y >= 0.0, ps(K["Ca"], K["Da"]), ps(K["Cb"], K["Db"]))


def U_s(c: Channel):
    """App. C: characteristic thermocapillary velocity on the interface."""
    r = c.a / c.b
    C1 = (c.T_h * r + c.T_c * c.k_ratio) / (r + c.k_ratio)
    C2 = c.dT * np.sinh(c.at) / (c.k_ratio * np.cosh(c.at) * np.sinh(c.bt) + np.cosh(c.bt) * np.sinh(c.at))
    return (c.dT / c.mu_b) * (c.b / c.l) * (c.sigma_T + 2.0 * c.sigma_TT * (C1 + C2 - c.T_ref))


def U_ygb(sigma_T, gradT, R, mu_b, k_ratio, mu_ratio):
    """Sec. 5.1: Young-Goldstein-Block terminal velocity of a droplet."""
    U_star = -sigma_T * abs(gradT) * R / mu_b
    return 2.0 * U_star / ((2.0 + k_ratio) * (2.0 + 3.0 * mu_ratio))


def sign_changes_periodic(v, tol=0.0):
    """Number of sign changes of a periodic sample (zeros within tol are skipped)."""
    s = np.sign(np.where(np.abs(v) <= tol, 0.0, v))
    s = s[s != 0]
    if s.size == 0:
        return 0
    return int(np.sum(s != np.roll(s, 1)))


def vortex_count(c: Channel, n: int = 4096):
    """Cells = sign changes of v along x at the mid-height of each layer, summed."""
    x = np.arange(n) * c.l / n
    total = 0
    for y in (-0.5 * c.b, 0.5 * c.a):
        _, v = velocity(c, x, np.full_like(x, y))
        total += sign_changes_periodic(v, tol=1e-12 * max(np.max(np.abs(v)), 1e-300))
    return total
