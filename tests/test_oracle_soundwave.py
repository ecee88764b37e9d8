"""Pins of the linear sound-wave initial conditions (Sec. 3.1) through the
FP64 oracle: the displacement dx = -(A/2 pi) cos(2 pi x - pi/2) of a BCC
lattice imprints rho = 1 + A cos(2 pi x) on the kernel-weighted density.
The kernel smooths a wave of wavenumber k by a factor 1 - O((k h)^2), so the
measured amplitude approaches A with second-order convergence: doubling N
(halving h) cuts the amplitude loss by four."""
import math

import numpy as np

import oracle
from paper_2511_11425_gb300 import inputs


def _fit(N):
    p = inputs.soundwave(N)
    op = oracle.Params(kernel=p.kernel, n_ngb=p.n_ngb, gamma=p.gamma, alpha=p.alpha,
                       beta=p.beta, box_lo=p.box_lo, box_hi=p.box_hi, periodic=p.periodic)
    sinks = np.random.default_rng(0).choice(p.n, 256, replace=False)
    d = oracle.density_h(op, p.pos, p.m, p.h0, sinks)
    assert d["failed"] == 0
    x = p.pos[sinks, 0]
    M = np.stack([np.ones_like(x), np.cos(2 * math.pi * x), np.sin(2 * math.pi * x)], 1)
    coef, *_ = np.linalg.lstsq(M, d["rho"], rcond=None)
    resid = float(np.std(d["rho"] - M @ coef))
    return p, coef, resid


def test_soundwave_density_wave_is_imprinted():
    p32, c32, r32 = _fit(32)
    p64, c64, r64 = _fit(64)
    A = p32.extra["A"]
    assert p32.n == 2 * 32 * 16 * 16 and p64.n == 2 * 64 * 16 * 16
    for c, r in ((c32, r32), (c64, r64)):
        assert abs(c[0] - 1.0) < 1e-4            # unit mean density
        assert abs(c[2]) < 1e-3 * A              # cosine phase: no sine part
        assert r < 1e-3 * A                      # nothing but the wave
        assert 0.98 * A < c[1] < A               # the kernel smooths it slightly
    loss32, loss64 = 1.0 - c32[1] / A, 1.0 - c64[1] / A
    assert 3.5 < loss32 / loss64 < 4.5           # smoothing loss ~ (k h)^2


def test_soundwave_pressure_and_velocity_follow_the_density():
    p = inputs.soundwave(16)
    A = p.extra["A"]
    x = p.pos[:, 0]
    P = (p.gamma - 1.0) * (1.0 + A * np.cos(2 * math.pi * x)) * p.u
    P0 = 1.0 / p.gamma
    assert np.allclose(P, P0 * (1.0 + p.gamma * A * np.cos(2 * math.pi * x)), rtol=1e-12)
    assert np.allclose(p.vel[:, 0], A * np.cos(2 * math.pi * x))   # c = sqrt(gamma P0) = 1
    assert math.isclose(math.sqrt(p.gamma * P0 / 1.0), 1.0)
