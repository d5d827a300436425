"""Pins of the closed-form solution (oracle/analytic.py) to the mathematics and to the
numbers the paper prints.  CPU only."""
import json
import os

import numpy as np
import pytest

from oracle import analytic as A

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.json")))


def _chan(**kw):
    base = dict(l=200.0, a=50.0, b=50.0, k_ratio=1.0, mu_ratio=1.0, mu_b=0.2,
                sigma_T=0.0, sigma_TT=0.0)
    base.update(kw)
    return A.Channel(**base)


GENERIC = [
    _chan(k_ratio=1.5, mu_ratio=2.0, sigma_T=-5e-4, sigma_TT=1e-3, T_h=1.2, T_c=1.0, T_ref=1.1),
    _chan(a=150.0, b=50.0, k_ratio=0.3, mu_ratio=0.5, sigma_T=2e-5, sigma_TT=-2e-4),
    _chan(a=20.0, b=60.0, l=128.0, k_ratio=4.0, mu_ratio=3.0, sigma_T=1e-4, sigma_TT=5e-4, T_h=2.0),
]


@pytest.mark.parametrize("c", GENERIC)
def test_no_slip_at_both_walls(c):
    x = np.linspace(0, c.l, 33)
    for y in (-c.b, c.a):
        u, v = A.velocity(c, x, np.full_like(x, y))
        scale = abs(A.U_t(c)) + abs(A.U_tt(c))
        assert np.max(np.abs(u)) <= 1e-12 * scale
        assert np.max(np.abs(v)) <= 1e-12 * scale


@pytest.mark.parametrize("c", GENERIC)
def test_interface_continuity_and_no_through_flow(c):
    x = np.linspace(0, c.l, 33)
    ua, va = A.velocity(c, x, np.zeros_like(x))
    ub, vb = A.velocity(c, x, np.full_like(x, -1e-300))
    expect = A.U_t(c) * np.sin(c.omega * x) + 0.5 * A.U_tt(c) * np.sin(2 * c.omega * x)
    scale = abs(A.U_t(c)) + abs(A.U_tt(c))
    assert np.max(np.abs(ua - expect)) <= 1e-12 * scale
    assert np.max(np.abs(ub - expect)) <= 1e-12 * scale
    assert np.max(np.abs(va)) <= 1e-12 * scale and np.max(np.abs(vb)) <= 1e-12 * scale


@pytest.mark.parametrize("c", GENERIC)
def test_marangoni_stress_balance(c):
    """mu_b du^b/dy - mu_a du^a/dy = (dsigma/dT) dT/dx at y = 0 (Sec. 3.2, condition v)."""
    x = np.linspace(0, c.l, 41)
    h = 1e-4 * c.b

    def d_dy(side):
        ys = side * np.array([0.0, h, 2 * h])
        if side < 0:
            ys[0] = -1e-300
        us = [A.velocity(c, x, np.full_like(x, y))[0] for y in ys]
        return side * (-3 * us[0] + 4 * us[1] - us[2]) / (2 * h)

    lhs = c.mu_b * d_dy(-1) - c.mu_b * c.mu_ratio * d_dy(+1)
    T0 = A.temperature(c, x, np.zeros_like(x))
    e = 1e-4
    dTdx = (A.temperature(c, x + e, np.zeros_like(x)) - A.temperature(c, x - e, np.zeros_like(x))) / (2 * e)
    rhs = (c.sigma_T + 2 * c.sigma_TT * (T0 - c.T_ref)) * dTdx
    assert np.max(np.abs(lhs - rhs)) <= 1e-6 * np.max(np.abs(rhs))


@pytest.mark.parametrize("c", GENERIC)
def test_velocity_divergence_free_and_stokes(c):
    """div u = 0 and the stream function is biharmonic in each layer (Sec. 3.2)."""
    rng = np.random.default_rng(1)
    e = 1e-3 * min(c.a, c.b)
    for layer in (-1, 1):
        x = rng.uniform(0, c.l, 20)
        y = layer * rng.uniform(0.1, 0.9, 20) * (c.a if layer > 0 else c.b)
        dudx = (A.velocity(c, x + e, y)[0] - A.velocity(c, x - e, y)[0]) / (2 * e)
        dvdy = (A.velocity(c, x, y + e)[1] - A.velocity(c, x, y - e)[1]) / (2 * e)
        du = np.max(np.abs(dudx)) + 1e-300
        assert np.max(np.abs(dudx + dvdy)) <= 1e-4 * du
        # u = dpsi/dy, v = -dpsi/dx
        dpsidy = (A.stream_function(c, x, y + e) - A.stream_function(c, x, y - e)) / (2 * e)
        assert np.max(np.abs(dpsidy - A.velocity(c, x, y)[0])) <= 1e-4 * np.max(np.abs(A.velocity(c, x, y)[0]))
        # biharmonic: nabla^4 psi ~ 0 relative to the terms it cancels
        hh = 0.05 * min(c.a, c.b) * 0.1
        P = lambda dx, dy: A.stream_function(c, x + dx * hh, y + dy * hh)
        lap = lambda dx, dy: (P(dx + 1, dy) + P(dx - 1, dy) + P(dx, dy + 1) + P(dx, dy - 1) - 4 * P(dx, dy)) / hh ** 2
        bih = (lap(1, 0) + lap(-1, 0) + lap(0, 1) + lap(0, -1) - 4 * lap(0, 0)) / hh ** 2
        ref = np.max(np.abs(lap(0, 0))) * c.omega ** 2
        assert np.max(np.abs(bih)) <= 2e-2 * ref


@pytest.mark.parametrize("c", GENERIC)
def test_temperature_boundary_and_interface_conditions(c):
    """App. A: wall temperatures, continuity of T and of the heat flux at y = 0, Laplace."""
    x = np.linspace(0, c.l, 37)
    Tb = A.temperature(c, x, np.full_like(x, -c.b))
    Ta = A.temperature(c, x, np.full_like(x, c.a))
    assert np.allclose(Tb, c.T_h + c.dT * np.cos(c.omega * x), atol=1e-13)
    assert np.allclose(Ta, c.T_c, atol=1e-13)
    e = 1e-5 * c.b
    up = A.temperature(c, x, np.full_like(x, 0.0))
    dn = A.temperature(c, x, np.full_like(x, -1e-300))
    assert np.allclose(up, dn, atol=1e-13)
    flux_a = c.k_ratio * (A.temperature(c, x, np.full_like(x, e)) - up) / e
    flux_b = (dn - A.temperature(c, x, np.full_like(x, -e))) / e
    assert np.max(np.abs(flux_a - flux_b)) <= 1e-4 * (np.max(np.abs(flux_b)) + 1e-12)
    # harmonic in each layer
    h = 0.5
    for y0 in (-0.5 * c.b, 0.5 * c.a):
        y = np.full_like(x, y0)
        lap = (A.temperature(c, x + h, y) + A.temperature(c, x - h, y) + A.temperature(c, x, y + h)
               + A.temperature(c, x, y - h) - 4 * A.temperature(c, x, y)) / h ** 2
        assert np.max(np.abs(lap)) <= 1e-3 * c.dT * c.omega ** 2


def test_normal_fluid_limit_has_no_second_harmonic():
    """sigma_TT = 0 recovers the single-harmonic (Pendse-Esmaeeli) solution (Sec. 3.2)."""
    c = _chan(sigma_T=-5e-4, sigma_TT=0.0)
    assert A.U_tt(c) == 0.0
    assert A.vortex_count(c) == 4


def test_printed_droplet_velocity():
    g = GOLD["ygb_droplet"]
    u = A.U_ygb(g["sigma_T"], g["gradT"], g["R"], g["mu_b"], g["k_ratio"], g["mu_ratio"])
    assert abs(u - g["U_ygb"]) <= g["rel_tol"] * g["U_ygb"]


@pytest.mark.parametrize("key", ["nf_channel_Ca", "srf_channel_Ca",
                                 "srf_deformation_Ca_M2_3", "srf_deformation_Ca_M2_5", "srf_deformation_Ca_M2_10", "srf_deformation_Ca_M2_20"])
def test_printed_capillary_numbers(key):
    """Ca = U_s mu_b / sigma0 with U_s of App. C reproduces the printed Ca (2 digits)."""
    g = GOLD[key]
    c = _chan(l=g["l"], a=g["a"], b=g["b"], sigma_T=g["M1"] * g["sigma0"], sigma_TT=g["M2"] * g["sigma0"])
    Ca = abs(A.U_s(c)) * c.mu_b / g["sigma0"]
    assert abs(Ca - g["Ca"]) <= g["rel_tol"] * g["Ca"] + 5e-5


@pytest.mark.parametrize("key", ["nf_channel_Ca", "srf_channel_Ca", "srf_mixed_small_M1", "srf_mixed_large_M1",
                                 "srf_deformation_Ca_M2_3", "srf_deformation_Ca_M2_5", "srf_deformation_Ca_M2_10", "srf_deformation_Ca_M2_20"])
def test_printed_vortex_counts_and_direction(key):
    g = GOLD[key]
    c = _chan(l=g["l"], a=g["a"], b=g["b"], sigma_T=g["M1"] * g["sigma0"], sigma_TT=g["M2"] * g["sigma0"])
    assert A.vortex_count(c) == g["vortices"]
    if "toward_hot_spot" in g:
        x = np.array([c.l / 16])
        u, _ = A.velocity(c, x, np.zeros(1))
        assert (u[0] < 0) == g["toward_hot_spot"]


def test_printed_thickness_ratio_effect():
    g = GOLD["thickness_ratio_effect"]
    x = np.linspace(0, 200, 801)
    umax = {}
    for ab in (1.0 / 3.0, 3.0):
        b = 100.0 / (1.0 + ab)
        c = _chan(a=100.0 - b, b=b, sigma_TT=0.1 * 1e-2)
        umax[ab] = np.max(np.abs(A.velocity(c, x, np.zeros_like(x))[0]))
    assert umax[3.0] >= g["ratio_min"] * umax[1.0 / 3.0]
