"""Pins of the oracle's interface correction (Sec. 2.3.4): the kernel
imbalance (Eq. Kernel_imbalance) and its normalisation, the exp(-I^2)
weighted averages of T and P, and the corrected density from the EOS."""
import os

import numpy as np
import pytest

import oracle
from paper_2511_11425_gb300 import inputs


def _golden():
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden",
                                  "interface_two_particles.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_imbalance_normalisation_closed_form():
    # Wendland C2: 2 pi int_0^1 (21/2pi)(1-q)^4 (1+4q) q^3 dq
    #            = 21 (B(4,5) + 4 B(5,5)) = 21 (1/280 + 1/157.5) = 5/24
    assert oracle.imbalance_norm("wc2") == pytest.approx(24.0 / 5.0, rel=1e-12)
    # Wendland C4: (495/16) (B(4,7) + 6 B(5,7) + 35/3 B(6,7)) = 35/192
    assert oracle.imbalance_norm("wc4") == pytest.approx(192.0 / 35.0, rel=1e-12)
    # Wendland C6: (1365/32) (B(4,9) + 8 B(5,9) + 25 B(6,9) + 32 B(7,9)) = 21/128
    assert oracle.imbalance_norm("wc6") == pytest.approx(128.0 / 21.0, rel=1e-12)
    # cubic spline: 16 (int_0^1/2 (q^3 - 6 q^5 + 6 q^6) dq + 2 int_1/2^1 (1-q)^3 q^3 dq)
    #             = 16 (3/448 + 1/140) = 31/140
    assert oracle.imbalance_norm("m4") == pytest.approx(140.0 / 31.0, rel=1e-12)


def test_two_particle_interface_correction_matches_hand_values():
    g = _golden()
    p = oracle.Params(kernel="wc2", gamma=5.0 / 3.0, box_lo=(-2, -2, -2), box_hi=(2, 2, 2),
                      periodic=(0, 0, 0))
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    out = oracle.interface_correction(p, pos, np.ones(2), np.ones(2), np.array([1.0, 0.25]),
                                      np.array([1.0, 3.0]), np.array([0, 1]), [1.0, 2.0])
    assert out["I"][0] == pytest.approx(g["I1"], rel=1e-11)
    assert out["I"][1] == pytest.approx(g["I2"], rel=1e-11)
    assert out["rho_corr"][0] == pytest.approx(g["rho_c1"], rel=1e-11)
    assert out["rho_corr"][1] == pytest.approx(g["rho_c2"], rel=1e-11)


def _layers(n=10):
    """Jittered periodic lattice split into two materials at z = 0.5 (and the
    periodic image of that plane at z = 0)."""
    prob = inputs.uniform(n=n, seed=61, jitter=0.02, vamp=0.0)
    prob.m = np.full(prob.n, 1.0 / prob.n)      # equal masses, uniform u: only the
    prob.u = np.ones(prob.n)                    # materials make an imbalance
    mat = (prob.pos[:, 2] >= 0.5).astype(np.int32)
    p = oracle.Params(gamma=prob.gamma, box_lo=prob.box_lo, box_hi=prob.box_hi,
                      periodic=prob.periodic)
    d = oracle.density_h(p, prob.pos, prob.m, prob.h0)
    return prob, p, mat, d


def test_imbalance_vanishes_inside_one_material_and_is_one_at_an_interface():
    prob, p, mat, d = _layers()
    one = oracle.imbalance(p, prob.pos, prob.m, d["h"], np.zeros(prob.n, dtype=np.int32))
    assert np.max(one) < 0.05                        # a single material: no imbalance
    I = oracle.imbalance(p, prob.pos, prob.m, d["h"], mat)
    z = prob.pos[:, 2]
    dist = np.minimum(np.abs(z - 0.5), np.minimum(z, 1.0 - z))  # to the nearest interface
    dx = 1.0 / 10
    near = dist < 0.6 * dx                            # the two layers next to an interface
    far = dist > 0.95 * np.max(d["h"])          # the kernel does not reach the other side
    # normalised so that a particle on a flat interface has I = 1; the
    # layers sit half a spacing off the plane
    assert 0.6 < np.min(I[near]) and np.max(I[near]) < 1.0, (I[near].min(), I[near].max())
    assert np.max(I[far]) < 0.05


def test_correction_leaves_a_single_material_alone():
    prob, p, mat, d = _layers()
    one = np.zeros(prob.n, dtype=np.int32)
    out = oracle.interface_correction(p, prob.pos, prob.m, d["h"], d["rho"], prob.u, one, [1.0])
    assert np.max(np.abs(out["rho_corr"] / d["rho"] - 1.0)) < 1e-4


def slab_problem(n=14):
    """Two ideal gases in pressure and temperature equilibrium: a slab
    0.25 < z < 0.75 of material 1 at density 2 (double particle mass, same
    lattice) in material 0 at density 1; P = 1, gas constants 1 and 1/2 so
    that T = P / (rho R) = 1 on both sides."""
    prob = inputs.uniform(n=n, seed=71, jitter=0.1, vamp=0.0)
    z = prob.pos[:, 2]
    mat = ((z > 0.25) & (z < 0.75)).astype(np.int32)
    rho_true = np.where(mat == 1, 2.0, 1.0)
    prob.m = rho_true / prob.n
    prob.u = 1.0 / ((prob.gamma - 1.0) * rho_true)
    prob.extra["mat"] = mat
    prob.extra["r_gas"] = (1.0, 0.5, 1.0, 1.0)
    prob.extra["rho_true"] = rho_true
    return prob


def test_correction_moves_the_density_towards_the_eos_at_an_isothermal_interface():
    prob = slab_problem()
    p = oracle.Params(gamma=prob.gamma, box_lo=prob.box_lo, box_hi=prob.box_hi,
                      periodic=prob.periodic)
    d = oracle.density_h(p, prob.pos, prob.m, prob.h0)
    ic = oracle.interface_correction(p, prob.pos, prob.m, d["h"], d["rho"], prob.u,
                                     prob.extra["mat"], prob.extra["r_gas"])
    rt = prob.extra["rho_true"]
    err_sum = np.abs(d["rho"] / rt - 1.0)
    err_ic = np.abs(ic["rho_corr"] / rt - 1.0)
    # the kernel sum smooths the jump over h; the corrected density takes
    # P and T from the particles away from the interface
    assert np.max(err_ic) < 0.75 * np.max(err_sum)
    assert np.mean(err_ic) < 0.75 * np.mean(err_sum)
    # away from the interface nothing changes
    z = prob.pos[:, 2]
    far = (np.abs(z - 0.25) > 1.05 * np.max(d["h"])) & (np.abs(z - 0.75) > 1.05 * np.max(d["h"]))
    assert np.max(np.abs(ic["rho_corr"][far] / d["rho"][far] - 1.0)) < 1e-3
