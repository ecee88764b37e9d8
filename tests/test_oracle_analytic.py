"""Pins for the analytic solutions the paper compares against (Sec. 3.2 Sod
tube, Sec. 3.3 Sedov-Taylor blast): published constants in tests/golden/."""
import os

import numpy as np

from oracle import riemann, sedov

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_sod_star_state_matches_toro():
    g = _read("toro_sod_star.txt")
    s = riemann.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert abs(s["p"] - g["p_star"]) < 1e-5
    assert abs(s["u"] - g["u_star"]) < 1e-5
    assert abs(s["rhoL"] - g["rho_star_L"]) < 1e-5
    assert abs(s["rhoR"] - g["rho_star_R"]) < 1e-5
    assert abs(s["SR"] - g["shock_speed"]) < 1e-5


def test_riemann_sample_limits():
    xi = np.array([-10.0, 10.0])
    rho, u, p = riemann.sample(xi, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert np.allclose(rho, [1.0, 0.125]) and np.allclose(p, [1.0, 0.1]) and np.allclose(u, 0)
    # the rarefaction fan is continuous at its tail
    s = riemann.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    r2, u2, p2 = riemann.sample(np.array([s["SL_tail"] - 1e-9]), 1.0, 0.0, 1.0, 0.125, 0.0,
                                0.1, 1.4)
    assert abs(p2[0] - s["p"]) < 1e-6 and abs(u2[0] - s["u"]) < 1e-6


def test_sedov_constants():
    g = _read("sedov_constants.txt")
    s53 = sedov.SedovSolution(5.0 / 3.0)
    assert abs(s53.xi0 - g["xi0_gamma_5_3"]) < 2e-5
    assert abs(sedov.SedovSolution(1.4).xi0 - g["xi0_gamma_1_4"]) < 1e-3
    rho, v, P = s53.profile(np.array([0.999999 * s53.shock_radius(0.05)]), 0.05)
    assert abs(rho[0] - g["density_jump_5_3"]) < 1e-3
    # shock radius at t = 0.05 for E = rho0 = 1
    assert abs(s53.shock_radius(0.05) - 1.15167 * 0.05 ** 0.4) < 1e-4


def test_sedov_profile_conserves_energy():
    s = sedov.SedovSolution(5.0 / 3.0)
    t = 0.05
    R = s.shock_radius(t)
    r = np.linspace(1e-4, R * (1 - 1e-9), 200001)
    rho, v, P = s.profile(r, t)
    e = (0.5 * rho * v * v + P / (s.gamma - 1.0)) * 4 * np.pi * r * r
    assert abs(np.trapezoid(e, r) - 1.0) < 2e-3
