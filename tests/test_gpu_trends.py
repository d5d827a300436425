"""The paper's parametric study (Sec. 6): U_max on the interface against k~ and mu~ for
a/b = 1/3, 1, 3, and against M2, run as one batched FP64 sweep to steady state and compared
with the closed-form solution of Sec. 3 (the oracle's analytic module, read at the same two
node rows that straddle the interface).  The trends the paper describes are asserted
exactly; the LB-to-closed-form ratio within the band the finite interface width allows."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def analytic_u_max(c):
    from oracle import analytic as A
    d, p = c["domain"], c["params"]
    ch = A.Channel(l=d["nx"], a=d["ny"] - d["b"], b=d["b"], k_ratio=p["cond_ratio"], mu_ratio=p["visc_ratio"],
                   mu_b=(p["tau_flow"] - 0.5) / 3.0, sigma_T=p["sigma1"], sigma_TT=p["sigma2"],
                   T_h=p["T_hot"], T_c=p["T_cold"], T_ref=p["T_ref"], dT=p["dT"])
    x = np.arange(d["nx"], dtype=float)
    u_lo, _ = A.velocity(ch, x, np.full_like(x, -0.5))
    u_hi, _ = A.velocity(ch, x, np.full_like(x, 0.5))
    return float(np.max(np.abs(0.5 * (u_lo + u_hi))))


@pytest.mark.timeout(900)
def test_u_max_trends_match_closed_form():
    from paper_2210_07501_gb300 import trends as T
    ks, mus, m2s = (0.25, 1.0, 4.0), (0.25, 4.0), (2.5e-2, 1e-1)
    cl = T.cases("cond_ratio", ks) + T.cases("visc_ratio", mus) + T.cases("M2", m2s, ab_values=(1.0,))
    res, seconds = T.run(cl)
    print(f"sweep of {len(cl)} channels: {seconds:.1f} s")
    ratios = {}
    for c, r in zip(cl, res):
        ua = analytic_u_max(c)
        ratios[r["name"]] = r["U_lb"] / ua
        print(f"{r['name']:32s} steps {r['steps']:6d} conv {r['converged']} U_lb {r['U_lb']:.4e} "
              f"analytic {ua:.4e} ratio {r['U_lb'] / ua:.3f}")
    # LB vs the sharp-interface closed form at W = 5 on 200 x 100: measured 0.82 (k~ = 1/4)
    # .. 0.88 (base) .. 1.07 (k~ = 4); the diffuse interface costs ~10 %, as the oracle's own
    # Marangoni pin shows (20 % at 64 x 32, halving under refinement)
    for name, q in ratios.items():
        assert 0.78 <= q <= 1.10, (name, q)
    U = {r["name"]: r["U_lb"] for r in res}
    for ab in ("0.333", "1", "3"):
        k = [U[f"trend-ab={ab},cond_ratio={v:g}"] for v in ks]
        assert k[0] > k[1] > k[2]                                  # U_max falls with k~
        m = [U[f"trend-ab={ab},visc_ratio={v:g}"] for v in mus]
        assert m[0] < U[f"trend-ab={ab},cond_ratio=1"] < m[1]      # and rises with mu~
    # larger a/b (interface nearer the heated wall): faster, at every k~
    for v in ks:
        assert U[f"trend-ab=0.333,cond_ratio={v:g}"] < U[f"trend-ab=1,cond_ratio={v:g}"] < U[f"trend-ab=3,cond_ratio={v:g}"]
    # U_max is linear in M2 at M1 = 0
    u25, u50, u100 = U["trend-ab=1,M2=0.025"], U["trend-ab=1,cond_ratio=1"], U["trend-ab=1,M2=0.1"]
    assert abs(u50 / u25 - 2.0) < 0.02 and abs(u100 / u50 - 2.0) < 0.02


@pytest.mark.timeout(600)
def test_interface_deforms_more_at_larger_capillary_number():
    """Sec. 6, last study: a/b = 3, M2 = 3 .. 20 (Ca = 0.34 .. 2.29 by the analytic U_s, which
    reproduces the printed ladder): the interface deflects more as Ca grows, the layer
    volume is kept (mean height b), and the eight cells of the SRF layers persist."""
    from oracle import analytic as A
    from paper_2210_07501_gb300 import trends as T
    res, seconds = T.run_deformation()
    print(f"deformation sweep: {seconds:.1f} s")
    for r in res:
        c = A.Channel(l=200, a=75, b=25, k_ratio=1, mu_ratio=1, mu_b=(1.17 - 0.5) / 3, sigma_T=0.0,
                      sigma_TT=r["M2"] * 1e-3)
        r["Ca"] = abs(A.U_s(c)) * c.mu_b / 1e-3
        print(f"{r['name']:20s} Ca {r['Ca']:.3f} steps {r['steps']:6d} conv {r['converged']} "
              f"deflection {r['deflection']:.3f} mean height {r['mean_height']:.3f} cells {r['cells']} "
              f"u_max {r['u_max']:.3e}")
    d = [r["deflection"] for r in res]
    assert all(r["cells"] == 8 for r in res)
    assert all(abs(r["mean_height"] - 25.0) < 0.5 for r in res)
    assert d[0] < 0.05                                   # Ca = 0.011: flat, the analytic regime
    assert all(d[i] < d[i + 1] for i in range(len(d) - 1))
    # measured deflections 0.013, 1.87, 2.85, 4.61, 6.61 lattice units: growing with Ca,
    # sublinearly (the deformed interface relieves part of the pressure difference)
    assert d[1] > 1.0 and d[-1] > 3 * d[1]
