"""Workload definitions and seeded synthetic inputs for the coupled LB step.

This module is the only one shared by the CUDA path's callers and the oracle's
callers.  It holds no arithmetic of the method: only domain sizes, parameter sets
and seeded random numbers (numpy PCG64).  Each side builds its own initial state
from these inputs.

The channel workloads restate the paper's setups (Sec. 2.1, Sec. 5.2, Sec. 6):
a periodic channel, bottom wall heated as T_hot + dT cos(2 pi k x / nx), top wall
at T_cold, interface at height b, surface tension
sigma(T) = sigma0 + sigma1 (T - T_ref) + sigma2 (T - T_ref)^2.
Relaxation times tau give nu = M_phi = alpha = (tau - 1/2)/3 in lattice units.
"""
from __future__ import annotations

import copy

import numpy as np

DEFAULT_PARAMS = dict(
    sigma0=1e-3, sigma1=0.0, sigma2=-1e-4,
    T_ref=1.0, T_hot=1.0, T_cold=1.0, dT=1.0,
    tau_flow=0.8, visc_ratio=1.0, tau_T=0.8, cond_ratio=1.0, tau_phi=0.8,
    rho_bottom=1.0, rho_top=1.0, Fx_ext=0.0, Fy_ext=0.0,
)


def _cfg(name, domain, **over):
    p = dict(DEFAULT_PARAMS)
    p.update(over)
    return {"name": name, "domain": dict(domain), "params": p}


# Plain two-layer SRF channel, 128 x 32, interface at 16, width 4, D2Q9 flow with
# D2Q5 phase-field and energy lattices, all relaxation times 0.8, 2000 steps.
SRF_128x32 = _cfg("srf-channel-128x32",
                  dict(nx=128, ny=32, b=16.0, W=4.0, heat_periods=1, q_phi=5, q_T=5))

# Steady-state channel 1024 x 256, a = b = 128, width 5, viscosity and conductivity
# ratios 2, sigma2 = -2e-4, sigma1 in {0, 2e-5}.
SRF_1024x256 = _cfg("srf-channel-1024x256",
                    dict(nx=1024, ny=256, b=128.0, W=5.0, heat_periods=1, q_phi=5, q_T=5),
                    sigma1=0.0, sigma2=-2e-4, visc_ratio=2.0, cond_ratio=2.0)

# Bandwidth workload: 8192 x 2048 (16.8M sites), a/b = 0.5 (b = 1365, a = 683),
# four heating periods, width 5, otherwise as the 128 x 32 channel.
SRF_8192x2048 = _cfg("srf-channel-8192x2048",
                     dict(nx=8192, ny=2048, b=1365.0, W=5.0, heat_periods=4, q_phi=5, q_T=5))

# The paper's validation channels (Sec. 5.2 normal fluid, Sec. 6 self-rewetting):
# l = 200, a = b = 50, W = 5, M_phi = 0.02, sigma0 = 1e-2, k~ = mu~ = 1,
# T_h = T_c = T_ref = dT = 1.  nu and alpha are not printed; tau_flow and tau_T are
# chosen so that Re and Ma come out as printed (nu ~ 0.2, alpha ~ 0.8 for Sec. 5.2;
# nu ~ 0.22, alpha ~ 0.74 for Sec. 6).
PAPER_NF_200x100 = _cfg("paper-nf-channel-200x100",
                        dict(nx=200, ny=100, b=50.0, W=5.0, heat_periods=1, q_phi=9, q_T=9),
                        sigma0=1e-2, sigma1=-5e-4, sigma2=0.0, tau_phi=0.56,
                        tau_flow=1.1, tau_T=2.96)
PAPER_SRF_200x100 = _cfg("paper-srf-channel-200x100",
                         dict(nx=200, ny=100, b=50.0, W=5.0, heat_periods=1, q_phi=9, q_T=9),
                         sigma0=1e-2, sigma1=0.0, sigma2=1e-3, tau_phi=0.56,
                         tau_flow=1.17, tau_T=2.73)

# The paper's droplet case (Sec. 5.1): a 2-D drop of radius R = 20 at the centre of an
# 8R x 16R box, periodic in x, no-slip walls at T = 0 (bottom) and T = 32 (top), i.e. a
# uniform far-field gradient of 0.1; rho = c_p = 1, mu = k = 0.2 in both fluids, T_ref = 16,
# sigma0 = 2.5e-3, sigma_T = -1e-4.  nu = alpha = 0.2 give tau = 3 (0.2) + 1/2 = 1.1.  W and
# M_phi are not printed for this case: W = 5 and M_phi = 0.02 (tau_phi = 0.56) as in Sec. 5.2.
# The domain's b only feeds the default layer initialisation, which this case replaces.
PAPER_DROP_160x320 = _cfg("paper-drop-migration-160x320",
                          dict(nx=160, ny=320, b=160.0, W=5.0, heat_periods=1, q_phi=9, q_T=9),
                          sigma0=2.5e-3, sigma1=-1e-4, sigma2=0.0, T_ref=16.0, T_hot=0.0, T_cold=32.0,
                          dT=0.0, tau_flow=1.1, tau_T=1.1, tau_phi=0.56)
DROP_RADIUS = 20.0

WORKLOADS = {w["name"]: w for w in (SRF_128x32, SRF_1024x256, SRF_8192x2048,
                                     PAPER_NF_200x100, PAPER_SRF_200x100, PAPER_DROP_160x320)}


def workload(name: str, **domain_over) -> dict:
    """A deep copy of a named workload; keyword overrides go to the domain or params."""
    w = copy.deepcopy(WORKLOADS[name])
    for k, v in domain_over.items():
        if k in w["domain"]:
            w["domain"][k] = v
        else:
            w["params"][k] = v
    return w


def channel(nx, ny, b, W=4.0, heat_periods=1, q_phi=5, q_T=5, **params) -> dict:
    """An ad-hoc channel workload with DEFAULT_PARAMS overridden by ``params``."""
    return _cfg(f"channel-{nx}x{ny}", dict(nx=nx, ny=ny, b=float(b), W=float(W),
                                           heat_periods=heat_periods, q_phi=q_phi, q_T=q_T), **params)


def random_fields(nx: int, ny: int, seed: int, u_amp=1e-3, T_amp=0.2, dp_amp=1e-4,
                  phi_amp=0.05, modes=4) -> dict:
    """Seeded smooth random macroscopic fields (a few random Fourier modes each).

    Returns arrays of shape [ny][nx]: 'phi_pert' (added to the tanh interface by the
    caller's own initialisation, here only the perturbation), 'u', 'v', 'T_pert',
    'dp'.  Pure random numbers: no method arithmetic.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.arange(nx)[None, :]
    y = (np.arange(ny) + 0.5)[:, None]

    def smooth(amp):
        f = np.zeros((ny, nx))
        for _ in range(modes):
            kx = rng.integers(1, 4)
            ky = rng.integers(1, 4)
            ph1, ph2 = rng.uniform(0, 2 * np.pi, 2)
            c = rng.normal()
            f += c * np.cos(2 * np.pi * kx * x / nx + ph1) * np.sin(np.pi * ky * y / ny + ph2)
        return amp * f / max(1.0, np.sqrt(modes))

    return {"phi_pert": smooth(phi_amp), "u": smooth(u_amp), "v": smooth(u_amp),
            "T_pert": smooth(T_amp), "dp": smooth(dp_amp)}


def drop_fields(nx: int, ny: int, R: float, W: float, T_bottom: float, T_top: float,
                xc=None, yc=None) -> dict:
    """Initial fields of a drop case: phi = 1 inside a circle of radius R centred at
    (xc, yc) (default: the box centre) with a tanh edge of width W, the conduction profile
    between the wall temperatures (walls half a node outside the first and last rows), the
    fluid at rest and dp = 0.  Arrays [ny][nx]; node (i, j) sits at (i, j + 1/2)."""
    xc = nx / 2.0 if xc is None else xc
    yc = ny / 2.0 if yc is None else yc
    x = np.arange(nx)[None, :] + 0.0
    y = np.arange(ny)[:, None] + 0.5
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    phi = 0.5 + 0.5 * np.tanh(2.0 * (R - r) / W)
    T = np.broadcast_to(T_bottom + (T_top - T_bottom) * y / ny, (ny, nx)).copy()
    z = np.zeros((ny, nx))
    return {"phi": phi, "u": z, "v": z.copy(), "T": T, "dp": z.copy()}


def sweep_cases(n_cases: int = 96, seed: int = 0) -> list:
    """Seeded uneven parameter sweep: Lx in {256,512,1024}, Ly in {64,128,256},
    sigma1 ~ U[-2e-5, 2e-5], sigma2 ~ U[-4e-4, 0], a/b ~ U[0.25, 4],
    k~ ~ U[0.5, 4], mu~ ~ U[0.5, 4]; W = 5, tau = 0.8."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_cases):
        nx = int(rng.choice([256, 512, 1024]))
        ny = int(rng.choice([64, 128, 256]))
        s1 = float(rng.uniform(-2e-5, 2e-5))
        s2 = float(rng.uniform(-4e-4, 0.0))
        ab = float(rng.uniform(0.25, 4.0))
        kr = float(rng.uniform(0.5, 4.0))
        mr = float(rng.uniform(0.5, 4.0))
        b = float(round(ny / (1.0 + ab)))
        out.append(_cfg(f"sweep-{seed}-{i}", dict(nx=nx, ny=ny, b=b, W=5.0, heat_periods=1,
                                                   q_phi=5, q_T=5),
                        sigma1=s1, sigma2=s2, cond_ratio=kr, visc_ratio=mr))
    return out


def surrogate_cases(n_cases: int, seed: int, nx: int = 256, ny: int = 64) -> list:
    """The sweep's parameter distribution on one fixed grid (the warm-start surrogate's
    training and test channels; 256 x 64 by default): sigma1 ~ U[-2e-5, 2e-5],
    sigma2 ~ U[-4e-4, 0], a/b ~ U[0.25, 4], k~ ~ U[0.5, 4], mu~ ~ U[0.5, 4], W = 5, tau = 0.8."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_cases):
        s1 = float(rng.uniform(-2e-5, 2e-5))
        s2 = float(rng.uniform(-4e-4, 0.0))
        ab = float(rng.uniform(0.25, 4.0))
        kr = float(rng.uniform(0.5, 4.0))
        mr = float(rng.uniform(0.5, 4.0))
        b = float(min(max(round(ny / (1.0 + ab)), 3), ny - 3))
        out.append(_cfg(f"surrogate-{seed}-{i}", dict(nx=nx, ny=ny, b=b, W=5.0, heat_periods=1, q_phi=5, q_T=5),
                        sigma1=s1, sigma2=s2, cond_ratio=kr, visc_ratio=mr))
    return out
