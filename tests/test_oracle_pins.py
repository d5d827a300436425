"""Pins of the FP64 CPU oracle to what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign
or index, a transposed operand, a wrong relaxation rate) fails it:
  * App. B maps: P P^-1 = I, printed P^-1, F(u) against the brute-force definition of
    central moments, F(u) F(-u) = I;
  * Sec. 4.2 equilibrium against the matching principle (continuous Maxwellian central
    moments of rho c^2 plus phi_p times the lattice weights), source against the
    pressure/momentum it must inject, per-moment relaxation rates incl. the 2s/2d split;
  * macroscopic behaviour: exact mass conservation, stationary tanh interface of
    width W, diffusion of phi at M_phi, of T at alpha, shear decay at nu, Poiseuille,
    steady conduction against App. A, Marangoni convection against Sec. 3.2.
"""
import json
import os

import numpy as np
import pytest

import lbm_workloads as WL
from oracle import analytic as A

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
MOM = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (2, 1), (1, 2), (2, 2)]
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W5 = np.array([1 / 3] + [1 / 6] * 4)
C2 = 1.0 / 3.0


def central(pop, ux, uy):
    """Brute force: kappa_mn = sum_a pop_a (e_ax - ux)^m (e_ay - uy)^n."""
    Q = len(pop)
    return np.array([np.sum(pop * (EX[:Q] - ux) ** m * (EY[:Q] - uy) ** n) for (m, n) in MOM[:Q]])


def raw(pop):
    return central(pop, 0.0, 0.0)


# ---------------------------------------------------------------- App. B maps

@pytest.mark.parametrize("Q", [5, 9])
def test_P_inverse(oracle_mod, Q):
    P, Pi, _, _ = oracle_mod.matrices(Q, 0.0, 0.0)
    assert np.allclose(P @ Pi, np.eye(Q), atol=1e-15, rtol=0)
    assert np.allclose(Pi @ P, np.eye(Q), atol=1e-15, rtol=0)


def test_P_inverse_matches_printed(oracle_mod):
    printed = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "app_b_pinv.txt"))
    _, Pi, _, _ = oracle_mod.matrices(9, 0.0, 0.0)
    assert np.array_equal(Pi, printed)


@pytest.mark.parametrize("Q", [5, 9])
def test_F_is_central_moment_shift(oracle_mod, Q):
    rng = np.random.default_rng(3)
    for _ in range(5):
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        pop = rng.uniform(0, 1, Q)
        P, Pi, F, Fi = oracle_mod.matrices(Q, ux, uy)
        assert np.allclose(F @ (P @ pop), central(pop, ux, uy), atol=1e-14, rtol=0)
        assert np.allclose(F @ Fi, np.eye(Q), atol=1e-15, rtol=0)
        assert np.allclose(Pi @ (Fi @ central(pop, ux, uy)), pop, atol=1e-14, rtol=0)


# ---------------------------------------------------------------- Sec. 4.1 / 4.3 collisions

@pytest.mark.parametrize("Q", [5, 9])
def test_phase_collision_rates_and_conservation(oracle_mod, Q):
    rng = np.random.default_rng(5)
    w = W9 if Q == 9 else W5
    for _ in range(5):
        pop = rng.uniform(0, 0.3, Q)
        ux, uy = rng.uniform(-0.05, 0.05, 2)
        mx, my = rng.uniform(-0.01, 0.01, 2)
        om = rng.uniform(0.6, 1.8)
        phi = pop.sum()
        out = oracle_mod.collide_phase_site(pop, phi, ux, uy, mx, my, om)
        k0, k1 = central(pop, ux, uy), central(out, ux, uy)
        assert abs(out.sum() - phi) <= 1e-15
        assert np.allclose(k1[1:3], k0[1:3] + om * (np.array([mx, my]) - k0[1:3]), atol=1e-15)
        assert np.allclose(k1[3:5], C2 * phi, atol=1e-15)
        if Q == 9:
            assert np.allclose(k1[5:8], 0.0, atol=1e-15)
            assert abs(k1[8] - C2 * C2 * phi) <= 1e-15
    # rest equilibrium with no sharpening flux is phi times the lattice weights
    out = oracle_mod.collide_phase_site(np.zeros(Q), 0.7, 0.0, 0.0, 0.0, 0.0, 1.0)
    assert np.allclose(out, 0.7 * w, atol=1e-16)


@pytest.mark.parametrize("Q", [5, 9])
def test_energy_collision_rates(oracle_mod, Q):
    rng = np.random.default_rng(7)
    for _ in range(5):
        pop = rng.uniform(0, 0.4, Q)
        ux, uy = rng.uniform(-0.05, 0.05, 2)
        om = rng.uniform(0.6, 1.8)
        T = pop.sum()
        out = oracle_mod.collide_energy_site(pop, T, ux, uy, om)
        k0, k1 = central(pop, ux, uy), central(out, ux, uy)
        assert abs(out.sum() - T) <= 1e-15
        assert np.allclose(k1[1:3], (1 - om) * k0[1:3], atol=1e-15)
        assert np.allclose(k1[3:5], C2 * T, atol=1e-15)
        if Q == 9:   # matching the continuous Maxwellian with density T (Sec. 4.3)
            assert np.allclose(k1[5:8], 0.0, atol=1e-15)
            assert abs(k1[8] - C2 * C2 * T) <= 1e-15
        # first raw moment after a full relaxation carries T u (advection)
        out1 = oracle_mod.collide_energy_site(pop, T, ux, uy, 1.0)
        r = raw(out1)
        assert np.allclose(r[1:3], T * np.array([ux, uy]), atol=1e-15)


# ---------------------------------------------------------------- Sec. 4.2 flow collision

P0 = C2  # rho_A c^2 with rho_A = 1


def _matched_equilibrium_central(rho, p, ux, uy):
    """Matching principle: rho c^2 times the central moments of the continuous Maxwellian
    (1, 0, 0, c^2, c^2, 0, 0, 0, c^4) plus phi_p = p - rho c^2 times the lattice central
    moments of the weights (incompressible transformation)."""
    maxw = rho * C2 * np.array([1, 0, 0, C2, C2, 0, 0, 0, C2 * C2])
    return maxw + (p - rho * C2) * central(W9, ux, uy)


def test_flow_equilibrium_matching_principle(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(6):
        rho = rng.uniform(0.5, 2.0)
        dp = rng.uniform(-1e-3, 1e-3)
        ux, uy = rng.uniform(-0.05, 0.05, 2)
        gdev = rng.uniform(-1e-3, 1e-3, 9)
        out = oracle_mod.collide_flow_site(gdev, rho, dp, ux, uy, 0.0, 0.0, 0.0, 0.0, 1.0)
        g = out + W9 * P0
        p = P0 + dp
        # low-order raw moments (Sec. 4.2: pressure, momentum, momentum flux)
        r = raw(g)
        assert abs(r[0] - p) <= 1e-15
        assert np.allclose(r[1:3], rho * C2 * np.array([ux, uy]), atol=1e-16)
        assert abs(r[3] - C2 * (p + rho * ux * ux)) <= 1e-15
        assert abs(r[4] - C2 * (p + rho * uy * uy)) <= 1e-15
        assert abs(r[5] - C2 * rho * ux * uy) <= 1e-16
        # all central moments
        assert np.allclose(central(g, ux, uy), _matched_equilibrium_central(rho, p, ux, uy), atol=2e-16, rtol=0)


def test_flow_source_injects_pressure_and_force(oracle_mod):
    """With p = sum g + F_p.u/2 and rho c^2 u = sum g e + c^2 F_t/2 (Sec. 4.2), one
    collision adds F_p.u to sum g and c^2 F_t to sum g e, whatever the rates."""
    rng = np.random.default_rng(13)
    for _ in range(8):
        rho = rng.uniform(0.5, 2.0)
        gdev = rng.uniform(-1e-4, 1e-4, 9)
        Fp = rng.uniform(-1e-5, 1e-5, 2)
        Ft = rng.uniform(-1e-5, 1e-5, 2)
        om = rng.uniform(0.5, 1.9)
        r = raw(gdev)
        u = (r[1:3] + 0.5 * C2 * Ft) / (rho * C2)
        dp = r[0] + 0.5 * Fp @ u
        out = oracle_mod.collide_flow_site(gdev, rho, dp, u[0], u[1], Fp[0], Fp[1], Ft[0], Ft[1], om)
        r1 = raw(out)
        assert abs((r1[0] - r[0]) - Fp @ u) <= 1e-18
        assert np.allclose(r1[1:3] - r[1:3], C2 * Ft, atol=1e-18, rtol=0)


def _continuous_source_central(u, Fp, Ft, order=12):
    """Central moments (orders 00 .. 22, App. B order) of the continuous source of the
    pressure-based formulation (Sec. 4.2, incompressible transformation):
        S(xi) = (xi - u) . [ F_t G(xi; u) + F_p (G(xi; u) - G(xi; 0)) ],
    G(xi; m) the unit Gaussian of variance c^2 centred at m: the force term of the
    continuous Boltzmann equation for g = c^2 f + phi_p G(xi; 0).  Integrated by tensor
    Gauss-Hermite quadrature, exact for these polynomial-times-Gaussian integrands."""
    x, w = np.polynomial.hermite.hermgauss(order)
    s = np.sqrt(2.0 * C2)
    out = np.zeros(9)
    for centre, Fcoef in ((u, Ft + Fp), (np.zeros(2), -Fp)):
        X = centre[0] + s * x[:, None]
        Y = centre[1] + s * x[None, :]
        Wt = (w[:, None] * w[None, :]) / np.pi
        proj = (X - u[0]) * Fcoef[0] + (Y - u[1]) * Fcoef[1]
        for k, (m, n) in enumerate(MOM):
            out[k] += np.sum(Wt * proj * (X - u[0]) ** m * (Y - u[1]) ** n)
    return out


def test_flow_source_central_moments_match_continuous_source(oracle_mod):
    """The source's central moments sigma_mn of Sec. 4.2 (sigma_00 = Gamma, sigma_10,
    sigma_01, sigma_20, sigma_02, sigma_11), read off the oracle's collision, equal the
    central moments of the continuous forcing term through second order (the matching
    principle); the third- and fourth-order ones are zero as printed.  With every rate 1
    (omega_nu = 1) each post-collision central moment is equilibrium + sigma / 2, so the
    difference between a forced and an unforced collision of the same state is sigma / 2."""
    rng = np.random.default_rng(19)
    for _ in range(8):
        rho = rng.uniform(0.6, 1.8)
        ux, uy = rng.uniform(-0.08, 0.08, 2)
        Fp = rng.uniform(-1e-3, 1e-3, 2)
        Ft = rng.uniform(-1e-3, 1e-3, 2)
        dp = rng.uniform(-1e-3, 1e-3)
        gdev = rng.uniform(-1e-3, 1e-3, 9)
        forced = oracle_mod.collide_flow_site(gdev, rho, dp, ux, uy, Fp[0], Fp[1], Ft[0], Ft[1], 1.0)
        free = oracle_mod.collide_flow_site(gdev, rho, dp, ux, uy, 0.0, 0.0, 0.0, 0.0, 1.0)
        sigma = 2.0 * central(forced - free, ux, uy)
        cont = _continuous_source_central(np.array([ux, uy]), Fp, Ft)
        assert np.allclose(sigma[:6], cont[:6], atol=1e-17, rtol=1e-12), (sigma[:6], cont[:6])
        assert np.allclose(sigma[6:], 0.0, atol=1e-17), sigma[6:]
        # the matching is not vacuous: every second-order moment is present
        assert min(abs(cont[3]), abs(cont[4]), abs(cont[5])) > 1e-8


def test_flow_relaxation_rates_and_split(oracle_mod):
    """2s and all moments except 2d and 11 go to equilibrium; 2d and 11 relax at omega_nu."""
    rng = np.random.default_rng(17)
    for _ in range(6):
        rho = rng.uniform(0.8, 1.5)
        ux, uy = rng.uniform(-0.05, 0.05, 2)
        om = rng.uniform(0.5, 1.9)
        gdev = rng.uniform(-1e-3, 1e-3, 9)
        g = gdev + W9 * P0
        dp = g.sum() - P0
        p = P0 + dp
        eq = _matched_equilibrium_central(rho, p, ux, uy)
        k0 = central(g, ux, uy)
        out = oracle_mod.collide_flow_site(gdev, rho, dp, ux, uy, 0.0, 0.0, 0.0, 0.0, om)
        k1 = central(out + W9 * P0, ux, uy)
        # 2s -> equilibrium, 2d and 11 relax at omega
        assert abs((k1[3] + k1[4]) - (eq[3] + eq[4])) <= 1e-15
        d0, dq = k0[3] - k0[4], eq[3] - eq[4]
        assert abs((k1[3] - k1[4]) - (d0 + om * (dq - d0))) <= 1e-15
        assert abs(k1[5] - (k0[5] + om * (eq[5] - k0[5]))) <= 1e-15
        for m in (0, 1, 2, 6, 7, 8):
            assert abs(k1[m] - eq[m]) <= 1e-15


# ---------------------------------------------------------------- macroscopic pins

def _oracle(oracle_mod, w):
    return oracle_mod.Oracle(w["domain"], w["params"])


def test_mass_conserved_to_roundoff(oracle_mod):
    w = WL.channel(48, 24, 12, W=4.0, sigma0=1e-3, sigma1=2e-4, sigma2=-5e-4)
    o = _oracle(oracle_mod, w)
    rnd = WL.random_fields(48, 24, seed=21)
    y = np.arange(24)[:, None] + 0.5
    phi = 0.5 + 0.5 * np.tanh(2 * (y - 12) / 4.0) + rnd["phi_pert"] * 0
    o.init(phi=np.broadcast_to(phi, (24, 48)), u=rnd["u"], v=rnd["v"], T=1.0 + rnd["T_pert"], dp=rnd["dp"])
    m0 = o.mass()
    o.step(1500)
    assert abs(o.mass() - m0) <= 1e-13 * m0


@pytest.mark.parametrize("q", [5, 9])
def test_flat_interface_is_stationary(oracle_mod, q):
    """theta = 4 phi (1-phi)/W makes the tanh profile of width W the equilibrium (Sec. 3)."""
    w = WL.channel(16, 48, 24, W=5.0, q_phi=q, q_T=q, sigma0=0.0, sigma1=0.0, sigma2=0.0, dT=0.0)
    o = _oracle(oracle_mod, w)
    phi0 = o.fields()["phi"].copy()
    o.step(1000)
    phi1 = o.fields()["phi"].copy()
    o.step(1000)
    fl = o.fields()
    # the discrete profile settles within a few 1e-3 of the tanh and then stays put
    assert np.max(np.abs(fl["phi"] - phi0)) <= 1e-2
    assert np.max(np.abs(fl["phi"] - phi1)) <= 1e-9
    assert np.max(np.abs(fl["u"])) == 0.0 and np.max(np.abs(fl["v"])) == 0.0


def test_interface_relaxes_to_width_W(oracle_mod):
    """A profile twice too wide sharpens towards width W; a wrong sign of theta widens it."""
    ny, b, W = 64, 32.0, 4.0
    w = WL.channel(8, ny, b, W=W, sigma0=0.0, sigma1=0.0, sigma2=0.0, dT=0.0, tau_phi=1.0)
    o = _oracle(oracle_mod, w)
    y = np.arange(ny)[:, None] + 0.5
    wide = 0.5 + 0.5 * np.tanh(2 * (y - b) / (2 * W)) * np.ones((1, 8))
    o.init(phi=wide)
    target = 0.5 + 0.5 * np.tanh(2 * (y[:, 0] - b) / W)
    e0 = np.max(np.abs(wide[:, 0] - target))
    o.step(3000)
    e1 = np.max(np.abs(o.fields()["phi"][:, 0] - target))
    assert e1 <= 0.05 * e0


@pytest.mark.parametrize("q", [5, 9])
def test_phase_field_diffuses_at_mobility(oracle_mod, q):
    """With W -> infinity (theta -> 0) the Allen-Cahn lattice is diffusion at M_phi (Sec. 4.1)."""
    nx, ny, tau = 64, 4, 0.9
    w = WL.channel(nx, ny, 2, W=1e12, q_phi=q, q_T=q, sigma0=0.0, sigma1=0.0, sigma2=0.0, dT=0.0, tau_phi=tau)
    o = _oracle(oracle_mod, w)
    x = np.arange(nx)[None, :]
    amp = 1e-2
    o.init(phi=0.5 + amp * np.cos(2 * np.pi * x / nx) * np.ones((ny, 1)))
    steps = 400
    o.step(steps)
    phi = o.fields()["phi"]
    a1 = 2 * np.mean((phi - 0.5) * np.cos(2 * np.pi * x / nx))
    M = (tau - 0.5) / 3
    k = 2 * np.pi / nx
    measured = -np.log(a1 / amp) / (k * k * steps)
    assert abs(measured - M) <= 0.01 * M


@pytest.mark.parametrize("q", [5, 9])
def test_temperature_diffuses_at_alpha(oracle_mod, q):
    nx, ny, tau = 4, 32, 1.2
    w = WL.channel(nx, ny, 16, W=4.0, q_phi=q, q_T=q, sigma0=0.0, sigma1=0.0, sigma2=0.0, dT=0.0,
                   tau_T=tau, cond_ratio=1.0)
    o = _oracle(oracle_mod, w)
    y = np.arange(ny)[:, None] + 0.5
    amp = 0.1
    o.init(T=1.0 + amp * np.sin(np.pi * y / ny) * np.ones((1, nx)))
    steps = 300
    o.step(steps)
    T = o.fields()["T"][:, 0]
    a1 = 2 * np.mean((T - 1.0) * np.sin(np.pi * y[:, 0] / ny))
    alpha = (tau - 0.5) / 3
    k = np.pi / ny
    measured = -np.log(a1 / amp) / (k * k * steps)
    assert abs(measured - alpha) <= 0.01 * alpha


def test_shear_mode_decays_at_nu(oracle_mod):
    """u_x = A sin(pi y / H) between no-slip walls decays at nu (pi/H)^2 (omega_11, Sec. 4.2)."""
    nx, ny, tau = 4, 32, 0.9
    w = WL.channel(nx, ny, 16, W=4.0, sigma0=0.0, sigma1=0.0, sigma2=0.0, dT=0.0, tau_flow=tau)
    o = _oracle(oracle_mod, w)
    y = np.arange(ny)[:, None] + 0.5
    amp = 1e-4
    o.init(u=amp * np.sin(np.pi * y / ny) * np.ones((1, nx)))
    steps = 300
    o.step(steps)
    u = o.fields()["u"][:, 0]
    a1 = 2 * np.mean(u * np.sin(np.pi * y[:, 0] / ny))
    nu = (tau - 0.5) / 3
    k = np.pi / ny
    measured = -np.log(a1 / amp) / (k * k * steps)
    assert abs(measured - nu) <= 0.01 * nu


def test_poiseuille_profile(oracle_mod):
    """Uniform body force F_ext (Sec. 3, F_t = F_s + F_ext) between no-slip walls:
    u = F y (H - y) / (2 mu) with the walls halfway between nodes."""
    nx, ny, tau, F = 4, 24, 1.0, 1e-6
    w = WL.channel(nx, ny, 12, W=4.0, sigma0=0.0, sigma1=0.0, sigma2=0.0, dT=0.0, tau_flow=tau, Fx_ext=F)
    o = _oracle(oracle_mod, w)
    o.step(6000)
    u = o.fields()["u"][:, 0]
    y = np.arange(ny) + 0.5
    mu = (tau - 0.5) / 3
    exact = F * y * (ny - y) / (2 * mu)
    assert np.max(np.abs(u - exact)) <= 2e-3 * np.max(exact)


def _steady_conduction(oracle_mod, nx, ny, b, k_ratio=1.0):
    w = WL.channel(nx, ny, b, W=2.0, sigma0=0.0, sigma1=0.0, sigma2=0.0, tau_T=1.5, cond_ratio=k_ratio,
                   T_hot=1.0, T_cold=0.5, dT=0.5)
    o = _oracle(oracle_mod, w)
    o.step(int(6.0 * ny * ny))
    T = o.fields()["T"]
    c = A.Channel(l=nx, a=ny - b, b=b, k_ratio=k_ratio, mu_ratio=1.0, mu_b=0.1, sigma_T=0, sigma_TT=0,
                  T_h=1.0, T_c=0.5, T_ref=1.0, dT=0.5)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny) + 0.5 - b)
    Ta = A.temperature(c, X, Y)
    return np.sqrt(np.mean((T - Ta) ** 2))


def test_conduction_matches_appendix_A_second_order(oracle_mod):
    e1 = _steady_conduction(oracle_mod, 32, 16, 8)
    e2 = _steady_conduction(oracle_mod, 64, 32, 16)
    assert e2 <= 5e-4
    assert e1 / e2 >= 3.5      # second order under refinement (measured 3.9)


def test_conduction_with_conductivity_ratio(oracle_mod):
    """k~ != 1: the diffuse conductivity gives an O(W/L) error against App. A."""
    e = _steady_conduction(oracle_mod, 64, 32, 16, k_ratio=3.0)
    assert e <= 5e-3


def _marangoni(oracle_mod, nx, ny, b, steps, **prm):
    w = WL.channel(nx, ny, b, W=4.0, tau_flow=1.0, tau_T=1.5, sigma0=1e-3, **prm)
    o = _oracle(oracle_mod, w)
    o.step(steps)
    fl = o.fields()
    p = w["params"]
    c = A.Channel(l=nx, a=ny - b, b=b, k_ratio=p["cond_ratio"], mu_ratio=p["visc_ratio"],
                  mu_b=(p["tau_flow"] - 0.5) / 3, sigma_T=p["sigma1"], sigma_TT=p["sigma2"])
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny) + 0.5 - b)
    ua, va = A.velocity(c, X, Y)
    return fl, ua, va, c


def _cells(v, rows):
    return sum(A.sign_changes_periodic(v[r], tol=1e-3 * np.max(np.abs(v))) for r in rows)


@pytest.mark.parametrize("kind", ["srf", "nf"])
def test_marangoni_convection_against_section_3(oracle_mod, kind):
    """Eight cells and flow towards the hot spot for a self-rewetting fluid (sigma_TT > 0),
    four cells and flow away for a normal fluid (sigma_T < 0); interface velocity within
    the diffuse-interface error of the closed form (which halves under refinement)."""
    prm = dict(sigma1=0.0, sigma2=1e-3) if kind == "srf" else dict(sigma1=-5e-4, sigma2=0.0)
    nx, ny, b = 64, 32, 16
    fl, ua, va, c = _marangoni(oracle_mod, nx, ny, b, 3000, **prm)
    assert _cells(fl["v"], (b // 2, b + (ny - b) // 2)) == (8 if kind == "srf" else 4)
    u_if = 0.5 * (fl["u"][b - 1] + fl["u"][b])
    toward = u_if[nx // 16] < 0
    assert toward == (kind == "srf")
    err = np.linalg.norm(fl["u"] - ua) / np.linalg.norm(ua)
    assert err <= 0.25


def test_laplace_law_static_drop(oracle_mod):
    """Capillary term of the CSF force (Sec. 3, read with kappa = -div n and delta_s =
    1.5 W |grad phi|^2): a 2-D drop of fluid B holds p_in - p_out = sigma / R."""
    n, R, sig = 64, 16.0, 1e-3
    w = WL.channel(n, n, n / 2, W=4.0, sigma0=sig, sigma1=0.0, sigma2=0.0, dT=0.0, tau_flow=1.0)
    o = _oracle(oracle_mod, w)
    x = np.arange(n)[None, :]
    y = np.arange(n)[:, None] + 0.5
    r = np.sqrt((x - n / 2) ** 2 + (y - n / 2) ** 2)
    o.init(phi=0.5 - 0.5 * np.tanh(2 * (r - R) / 4.0))
    o.step(3000)
    dp = o.fields()["dp"]
    jump = dp[n // 2, n // 2] - dp[2, 2]
    assert abs(jump - sig / R) <= 0.15 * sig / R      # measured 0.93 sigma/R at W = 4


# ---------------------------------------------------------------- streaming and walls

def _delta_state(o, lattice, a, j, i, val=1e-3):
    st = o.get_state()
    for k in ("f", "g", "h"):
        st[k][:] = 0.0
    st["dp"][:] = 0.0
    st[lattice][a, j, i] = val
    o.set_state(st)


@pytest.mark.parametrize("q", [5, 9])
def test_streaming_routes_populations(oracle_mod, q):
    """Pull streaming f(x, t+1) = f~(x - e) with periodic x; at the halfway walls the flow
    lattice bounces back (no slip), the phase field reflects specularly (free slip, no
    flux through the wall) and the energy lattice anti-bounces to the wall temperature
    taken at the point where the link crosses the wall (Sec. 5.1 boundary treatment)."""
    nx, ny = 8, 6
    w = WL.channel(nx, ny, 3, W=4.0, q_phi=q, q_T=q, T_ref=1.0, T_hot=1.0, T_cold=1.0, dT=0.0)
    o = _oracle(oracle_mod, w)
    opp = {a: int(np.flatnonzero((EX[:9] == -EX[a]) & (EY[:9] == -EY[a]))[0]) for a in range(9)}
    mir = {a: int(np.flatnonzero((EX[:9] == EX[a]) & (EY[:9] == -EY[a]))[0]) for a in range(9)}
    # interior and periodic wrap
    _delta_state(o, "g", 5, 2, nx - 1)
    s = o.streamed()["g"]
    assert s[5, 3, 0] == 1e-3 and np.count_nonzero(s) == 1
    # flow lattice, bottom wall: population leaving downwards comes back reversed
    for a in (4, 7, 8):
        _delta_state(o, "g", a, 0, 3)
        s = o.streamed()["g"]
        assert s[opp[a], 0, 3] == 1e-3 and np.count_nonzero(s) == 1
    # phase field, top wall: specular reflection keeps the tangential velocity
    for a in [x for x in (2, 5, 6) if x < q]:
        _delta_state(o, "f", a, ny - 1, 3)
        s = o.streamed()["f"]
        assert s[mir[a], ny - 1, 3 + EX[a]] == 1e-3 and np.count_nonzero(s) == 1
    # energy lattice: anti-bounce-back flips the sign (wall at T_ref)
    for a in [x for x in (4, 7, 8) if x < q]:
        _delta_state(o, "h", a, 0, 3)
        s = o.streamed()["h"]
        assert abs(s[opp[a], 0, 3] + 1e-3) <= 1e-18 and np.count_nonzero(np.abs(s) > 1e-18) == 1


def test_energy_wall_temperature_at_link_crossing(oracle_mod):
    """h_a = -h~_abar + 2 w_a T_w with T_w at x_i - e_ax / 2 on the heated wall."""
    nx, ny, q = 8, 6, 9
    w = WL.channel(nx, ny, 3, W=4.0, q_phi=q, q_T=q, T_ref=1.0, T_hot=1.0, T_cold=1.0, dT=0.5, heat_periods=1)
    o = _oracle(oracle_mod, w)
    st = o.get_state()
    st["h"][:] = 0.0
    o.set_state(st)
    s = o.streamed()["h"]
    x = np.arange(nx)
    w9 = W9
    for a in (2, 5, 6):
        Tw = 1.0 + 0.5 * np.cos(2 * np.pi * (x - 0.5 * EX[a]) / nx)
        expect = 2 * w9[a] * Tw - w9[a] * 1.0 - w9[a] * 1.0   # h' = -h~' - w Tref + 2 w Tw - w Tref, h~' = 0
        assert np.allclose(s[a, 0], 2 * w9[a] * (Tw - 1.0), atol=1e-16)
        assert np.allclose(s[a, 0], expect, atol=1e-16)


def test_sigma_gradient_exact_up_to_the_walls(oracle_mod):
    """Ghost rows T = 2 T_w - T_adj make the isotropic gradient of a linear sigma(T)
    exact on the wall rows of a steady linear conduction profile."""
    nx, ny = 8, 16
    w = WL.channel(nx, ny, 8, W=4.0, sigma0=1e-3, sigma1=2e-4, sigma2=0.0, T_ref=1.0, T_hot=2.0,
                   T_cold=1.0, dT=0.0, tau_T=1.5)
    o = _oracle(oracle_mod, w)
    o.step(3000)
    d = o.debug_fields()
    exact = 2e-4 * (1.0 - 2.0) / ny
    assert np.allclose(d["dsy"], exact, rtol=1e-9, atol=0)
    assert np.allclose(d["dsx"], 0.0, atol=1e-18)


@pytest.mark.parametrize("rho_top,visc_ratio,tol", [(2.0, 1.0, 0.02), (1.0, 2.0, 0.01)])
def test_two_layer_poiseuille(oracle_mod, rho_top, visc_ratio, tol):
    """Uniform body force through two layers: the steady profile is the sharp-interface
    two-layer Poiseuille solution up to the diffuse-interface error.  With a density
    ratio the pressure force of the incompressible transformation (Sec. 4.2) carries the
    correction: without it the error is 24 %, with its sign flipped 39 %, as read 0.9 %.
    With a viscosity ratio the profile pins mu(phi) (bottom phi = 0 is fluid A)."""
    nx, ny, b, F, tau = 4, 48, 24.0, 1e-6, 1.0
    w = WL.channel(nx, ny, b, W=3.0, sigma0=0.0, sigma1=0.0, sigma2=0.0, dT=0.0, tau_flow=tau,
                   visc_ratio=visc_ratio, rho_bottom=1.0, rho_top=rho_top, Fx_ext=F)
    o = _oracle(oracle_mod, w)
    o.step(12000)
    u = o.fields()["u"][:, 0]
    muA = (tau - 0.5) / 3
    muB = visc_ratio * muA
    H = ny
    C = (F * b * b / 2 / muA - F * (b * b - H * H) / 2 / muB) / (b / muA - (b - H) / muB)
    y = np.arange(ny) + 0.5
    exact = np.where(y < b, (-F * y * y / 2 + C * y) / muA, (-F * (y * y - H * H) / 2 + C * (y - H)) / muB)
    assert np.linalg.norm(u - exact) / np.linalg.norm(exact) <= tol
    assert np.max(np.abs(o.fields()["v"])) <= 1e-6 * np.max(exact)
