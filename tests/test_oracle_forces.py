"""Pins for the oracle's force pass (Sec. 2.3.5 momentum, PdV and artificial
viscosity equations; Sec. 2.3.6 time-step criteria)."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_11425_gb300 import inputs


def _evaluate(prob, p, vel=None, u=None, m=None, pos=None):
    pos = prob.pos if pos is None else pos
    m = prob.m if m is None else m
    d = oracle.density_h(p, pos, m, prob.h0)
    assert d["failed"] == 0
    f = oracle.forces(p, pos, prob.vel if vel is None else vel, m, d["h"], d["rho"],
                      d["omega"], prob.u if u is None else u)
    return d, f


def _params(prob, **kw):
    base = dict(gamma=prob.gamma, alpha=prob.alpha, beta=prob.beta, box_lo=prob.box_lo,
                box_hi=prob.box_hi, periodic=prob.periodic)
    base.update(kw)
    return oracle.Params(**base)


@pytest.fixture(scope="module")
def rnd():
    prob = inputs.uniform(n=8, seed=21, jitter=0.35, vamp=0.5)
    p = _params(prob)
    d, f = _evaluate(prob, p)
    return prob, p, d, f


def test_momentum_conserved(rnd):
    # pairwise antisymmetry of every term -> sum_i m_i a_i = 0
    prob, p, d, f = rnd
    tot = (prob.m[:, None] * f["a"]).sum(0)
    scale = (prob.m[:, None] * np.abs(f["a"])).sum(0)
    assert np.all(np.abs(tot) < 1e-13 * scale)


def test_energy_balance_identity(rnd):
    # sum_i m_i (v_i . a_i + du_i/dt|H + du_i/dt|Pi) = 0 exactly: the PdV and
    # viscous heating terms absorb the work done by the pressure and viscous
    # accelerations (the equations come from one Lagrangian).
    prob, p, d, f = rnd
    terms = prob.m * ((prob.vel * f["a"]).sum(1) + f["dudt_h"] + f["dudt_av"])
    scale = np.abs(prob.m * (prob.vel * f["a"]).sum(1)).sum()
    assert abs(terms.sum()) < 1e-12 * scale
    assert np.any(f["dudt_av"] > 0) and np.all(f["dudt_av"] >= 0)


def test_angular_momentum_conserved_open_box():
    prob = inputs.uniform(n=6, seed=23, jitter=0.35, vamp=0.5, periodic=(0, 0, 0))
    p = _params(prob)
    d, f = _evaluate(prob, p)
    torque = (prob.m[:, None] * np.cross(prob.pos, f["a"])).sum(0)
    scale = (prob.m * np.linalg.norm(prob.pos, axis=1) * np.linalg.norm(f["a"], axis=1)).sum()
    assert np.all(np.abs(torque) < 1e-13 * scale)


def test_galilean_invariance(rnd):
    prob, p, d, f = rnd
    V = np.array([3.0, -1.5, 0.25])
    f2 = oracle.forces(p, prob.pos, prob.vel + V, prob.m, d["h"], d["rho"], d["omega"], prob.u)
    for k in ("a", "dudt_h", "dudt_av", "divv"):
        ref = np.max(np.abs(f[k]))
        assert np.max(np.abs(f2[k] - f[k])) < 1e-11 * ref


def test_mass_scaling_invariance(rnd):
    # at fixed u, scaling every mass by s scales rho, P by s and leaves every
    # acceleration and du/dt unchanged
    prob, p, d, f = rnd
    s = 7.0
    d2, f2 = _evaluate(prob, p, m=prob.m * s)
    for k in ("a", "dudt_h", "dudt_av", "divv", "dt"):
        ref = np.max(np.abs(f[k]))
        assert np.max(np.abs(f2[k] - f[k])) < 1e-10 * ref


def test_perfect_lattice_is_static():
    pos_prob = inputs.uniform(n=8, seed=1, jitter=0.0, vamp=0.0)
    u = np.full(pos_prob.n, 1.3)
    m = np.full(pos_prob.n, pos_prob.extra["dx"] ** 3)
    p = _params(pos_prob)
    d, f = _evaluate(pos_prob, p, u=u, m=m)
    P = (p.gamma - 1) * d["rho"] * u
    # every pressure term cancels by the lattice's point symmetry
    scale = np.max(P / d["rho"] / d["h"])
    assert np.max(np.abs(f["a"])) < 1e-11 * scale
    assert np.max(np.abs(f["dudt_h"])) == 0.0 and np.max(np.abs(f["dudt_av"])) == 0.0
    # no acceleration and no approaching pairs: dt is the bare Courant value
    c = np.sqrt(p.gamma * (p.gamma - 1) * u)
    dt = p.eta_courant * d["h"] / ((1 + 0.6 * p.alpha) * c)
    assert np.allclose(f["dt"], dt, rtol=1e-12)


def _internal_energy(p, pos, m, K, h0):
    d = oracle.density_h(p, pos, m, h0)
    assert d["failed"] == 0
    u = K * d["rho"] ** (p.gamma - 1) / (p.gamma - 1)
    return float((m * u).sum()), d


def test_pressure_force_is_gradient_of_internal_energy():
    # With h tied to rho by the constant-mass constraint, the hydro acceleration
    # is exactly -(1/m_i) dE/dx_i for E = sum_k m_k u_k(rho_k) at fixed entropy
    # (u = K rho^(gamma-1)/(gamma-1)), Omega carrying the dh/dx terms.
    prob = inputs.uniform(n=6, seed=31, jitter=0.3, vamp=0.0, periodic=(0, 0, 0))
    p = _params(prob, alpha=0.0, beta=0.0)
    idx = np.arange(prob.n, dtype=np.uint64)
    K = 0.5 + inputs.uniform01(99, idx, 0)
    E0, d = _internal_energy(p, prob.pos, prob.m, K, prob.h0)
    u = K * d["rho"] ** (p.gamma - 1) / (p.gamma - 1)
    f = oracle.forces(p, prob.pos, np.zeros_like(prob.pos), prob.m, d["h"], d["rho"],
                      d["omega"], u)
    for i in (0, 107, 180):
        for ax in range(3):
            eps = 1e-6 * d["h"][i]
            pp = prob.pos.copy()
            pp[i, ax] += eps
            Ep, _ = _internal_energy(p, pp, prob.m, K, d["h"])
            pm = prob.pos.copy()
            pm[i, ax] -= eps
            Em, _ = _internal_energy(p, pm, prob.m, K, d["h"])
            fd = -(Ep - Em) / (2 * eps) / prob.m[i]
            scale = np.max(np.abs(f["a"]))
            assert abs(fd - f["a"][i, ax]) < 2e-6 * scale


def test_pdv_heating_is_compression_rate():
    # du_i/dt|H = (P_i/rho_i^2) drho_i/dt and div v_i = -(1/rho_i) drho_i/dt,
    # with drho/dt taken by moving all particles along v (h re-solved).
    prob = inputs.uniform(n=6, seed=33, jitter=0.3, vamp=0.7, periodic=(0, 0, 0))
    p = _params(prob)
    d = oracle.density_h(p, prob.pos, prob.m, prob.h0)
    f = oracle.forces(p, prob.pos, prob.vel, prob.m, d["h"], d["rho"], d["omega"], prob.u)
    eps = 1e-7
    dp = oracle.density_h(p, prob.pos + eps * prob.vel, prob.m, d["h"])
    dm = oracle.density_h(p, prob.pos - eps * prob.vel, prob.m, d["h"])
    drho = (dp["rho"] - dm["rho"]) / (2 * eps)
    P = (p.gamma - 1) * d["rho"] * prob.u
    want = P / d["rho"] ** 2 * drho
    assert np.max(np.abs(f["dudt_h"] - want)) < 1e-6 * np.max(np.abs(want))
    assert np.max(np.abs(f["divv"] + drho / d["rho"])) < 1e-6 * np.max(np.abs(drho / d["rho"]))


def _two_body(vx, alpha, beta, h=1.0):
    pos = np.array([[0.0, 0.0, 0.0], [0.4, 0.0, 0.0]])
    vel = np.array([[vx, 0.0, 0.0], [-vx, 0.0, 0.0]])
    p = oracle.Params(alpha=alpha, beta=beta, periodic=(0, 0, 0), box_hi=(10, 10, 10))
    m = np.array([1.0, 1.0])
    rho = np.array([2.0, 2.0])
    om = np.array([1.0, 1.0])
    hh = np.array([h, h])
    u = np.array([1.0, 1.0])
    return oracle.forces(p, pos, vel, m, hh, rho, om, u)


def test_viscosity_is_repulsive_and_switches_off_when_receding():
    base = _two_body(0.0, 1.0, 2.0)
    app = _two_body(0.5, 1.0, 2.0)
    rec = _two_body(-0.5, 1.0, 2.0)
    # receding pairs feel pressure only, identical to the static pair
    assert np.allclose(rec["a"], base["a"], rtol=0, atol=1e-15)
    assert np.all(rec["dudt_av"] == 0.0)
    # approaching: extra push apart (particle 0 sits at smaller x), heating > 0
    assert app["a"][0, 0] < base["a"][0, 0] and app["a"][1, 0] > base["a"][1, 0]
    assert np.all(app["dudt_av"] > 0.0)


def test_viscosity_velocity_scaling():
    # Pi = (-alpha cbar mu + beta mu^2)/rhobar with mu ~ v: the viscous
    # acceleration is linear in v for beta = 0 and quadratic for alpha = 0.
    b0 = _two_body(0.0, 0.0, 0.0)["a"][0, 0]
    lin1 = _two_body(0.1, 1.0, 0.0)["a"][0, 0] - b0
    lin2 = _two_body(0.2, 1.0, 0.0)["a"][0, 0] - b0
    quad1 = _two_body(0.1, 0.0, 1.0)["a"][0, 0] - b0
    quad2 = _two_body(0.2, 0.0, 1.0)["a"][0, 0] - b0
    assert abs(lin2 / lin1 - 2.0) < 1e-12
    assert abs(quad2 / quad1 - 4.0) < 1e-12


def test_unequal_smoothing_lengths_keep_momentum():
    # the viscous terms use symmetric averages (hbar, cbar, rhobar) so the pair
    # force stays antisymmetric even when h_i != h_j
    pos = np.array([[0.0, 0.0, 0.0], [0.3, 0.1, -0.05]])
    vel = np.array([[0.4, 0.0, 0.1], [-0.3, 0.2, 0.0]])
    p = oracle.Params(periodic=(0, 0, 0), box_hi=(10, 10, 10))
    f = oracle.forces(p, pos, vel, np.array([1.0, 2.5]), np.array([0.5, 0.9]),
                      np.array([1.5, 3.0]), np.array([0.9, 1.1]), np.array([1.0, 0.4]))
    tot = 1.0 * f["a"][0] + 2.5 * f["a"][1]
    assert np.max(np.abs(tot)) < 1e-14 * np.max(np.abs(f["a"]))


def test_timestep_shrinks_with_compression():
    app = _two_body(0.5, 1.0, 2.0)
    rec = _two_body(-0.5, 1.0, 2.0)
    assert np.all(app["dt"] < rec["dt"])


def test_courant_limit_scales_with_approach_speed():
    # Eq. (courant_condition): with c -> 0 and alpha = 0 the Courant step is
    # eta_C h / (0.6 beta |mu|) and mu is linear in the approach speed, so
    # doubling the speed halves the step (the acceleration limit is switched
    # off with a huge eta_a).
    pos = np.array([[0.0, 0.0, 0.0], [0.4, 0.0, 0.0]])
    p = oracle.Params(alpha=0.0, beta=2.0, eta_acc=1e12, periodic=(0, 0, 0),
                      box_hi=(10, 10, 10))
    args = (np.array([1.0, 1.0]), np.array([1.0, 1.0]), np.array([2.0, 2.0]),
            np.array([1.0, 1.0]), np.array([1e-14, 1e-14]))
    dts = []
    for vx in (0.1, 0.2):
        vel = np.array([[vx, 0.0, 0.0], [-vx, 0.0, 0.0]])
        dts.append(oracle.forces(p, pos, vel, *args)["dt"])
    assert np.allclose(dts[1] / dts[0], 0.5, rtol=1e-5)


def test_pdv_sum_conditioning_output():
    """vdw_abs (the sum of the magnitudes of the PdV terms, used to bound
    FP32 cancellation) equals |sum| when every term has one sign (a uniform
    expansion v = x: v_ij . r_ij > 0 and dW/dr <= 0) and bounds it in a
    random flow; a uniform translation has no terms at all."""
    prob = inputs.uniform(n=6, seed=35, jitter=0.3, vamp=0.0, periodic=(0, 0, 0))
    p = _params(prob)
    d = oracle.density_h(p, prob.pos, prob.m, prob.h0)
    hubble = prob.pos - 0.5
    f = oracle.forces(p, prob.pos, hubble, prob.m, d["h"], d["rho"], d["omega"], prob.u)
    S = -f["divv"] * d["omega"] * d["rho"]
    assert np.allclose(f["vdw_abs"], np.abs(S), rtol=1e-12)
    assert np.allclose(f["divv_scale"], np.abs(f["divv"]), rtol=1e-12)
    rng = np.random.default_rng(4)
    v = rng.normal(size=prob.pos.shape)
    f = oracle.forces(p, prob.pos, v, prob.m, d["h"], d["rho"], d["omega"], prob.u)
    S = -f["divv"] * d["omega"] * d["rho"]
    assert np.all(f["vdw_abs"] >= np.abs(S) * (1 - 1e-12))
    assert np.all(f["dudt_h_scale"] >= np.abs(f["dudt_h"]) * (1 - 1e-12))
    f = oracle.forces(p, prob.pos, np.ones_like(v), prob.m, d["h"], d["rho"], d["omega"], prob.u)
    assert np.all(f["vdw_abs"] == 0.0)


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    vals = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_two_particle_forces_match_hand_values():
    """Absolute size of every force term, including the viscosity's mu_ij
    (h-bar factor, eps h-bar^2 in the denominator), Pi_ij, its acceleration
    and heating, and the Courant limit (tests/golden/two_particle_forces.txt)."""
    g = _golden("two_particle_forces.txt")
    p = oracle.Params(kernel="wc2", gamma=5.0 / 3.0, alpha=1.0, beta=2.0, eps_av=0.01,
                      eta_courant=0.15, eta_acc=0.2, box_lo=(-1.0, -1.0, -1.0),
                      box_hi=(1.0, 1.0, 1.0), periodic=(0, 0, 0))
    pos = np.array([[0.0, 0.0, 0.0], [0.3, 0.0, 0.0]])
    vel = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    f = oracle.forces(p, pos, vel, np.array([0.01, 0.02]), np.array([1.0, 0.5]),
                      np.array([1.2, 0.8]), np.array([1.0, 1.0]), np.array([0.9, 0.9]))
    tol = 1e-12
    assert f["a"][0, 0] == pytest.approx(g["a1x"], rel=tol)
    assert f["a"][1, 0] == pytest.approx(g["a2x"], rel=tol)
    assert np.all(f["a"][:, 1:] == 0.0)
    for k, idx in (("dudt_h", 0), ("dudt_av", 0), ("divv", 0), ("dt", 0)):
        for i in (0, 1):
            assert f[k][i] == pytest.approx(g["%s%d" % (k, i + 1)], rel=tol), (k, i)


def test_three_particle_totals_match_hand_values():
    g = _golden("three_particle_totals.txt")
    x = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    v = np.array([[0, 2.0, 0], [0, 0, 3.0], [4.0, 0, 0]])
    t = oracle.conserved(x, v, np.array([1.0, 2.0, 0.5]), np.array([1.0, 2.0, 3.0]))
    want = [g[k] for k in ("M", "Px", "Py", "Pz", "Lx", "Ly", "Lz", "Ekin", "Eint")]
    assert np.allclose(t, want, rtol=0, atol=1e-14), (t, want)
