"""Sedov-Taylor point-blast similarity solution (test infrastructure).

Used to compare the blast-wave run with the analytic solution, as the paper
does for its Sedov-Taylor test (Sec. 3.3).  Derived from the Euler equations
of a spherically symmetric ideal gas: with the shock radius
R(t) = xi0 (E t^2 / rho0)^(1/5), Rdot = 2R/(5t), eta = r/R and
    v = Rdot phi(eta),  rho = rho0 psi(eta),  P = rho0 Rdot^2 pi(eta),
mass, momentum and entropy conservation become three ODEs in eta,
    (phi-eta) psi' + psi phi' + 2 psi phi / eta = 0
    (phi-eta) phi' + pi'/psi = 3/2 phi
    (phi-eta) (pi'/pi - gamma psi'/psi) = 3
integrated inward from the strong-shock (Rankine-Hugoniot) state at eta = 1,
    psi = (g+1)/(g-1), phi = 2/(g+1), pi = 2/(g+1).
xi0 follows from energy conservation,
    1 = (16 pi / 25) xi0^5 int_0^1 (psi phi^2 / 2 + pi/(g-1)) eta^2 d eta.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp


def _rhs(eta, y, g):
    phi, psi, pi_ = y
    D = phi - eta
    num = 1.5 * phi - 3.0 * pi_ / (psi * D) + 2.0 * g * pi_ * phi / (psi * eta * D)
    den = D - g * pi_ / (psi * D)
    dphi = num / den
    dpsi = -psi * (dphi + 2.0 * phi / eta) / D
    dpi = pi_ * (3.0 / D + g * dpsi / psi)
    return [dphi, dpsi, dpi]


class SedovSolution:
    def __init__(self, gamma: float = 5.0 / 3.0, eta_min: float = 1e-5):
        g = gamma
        self.gamma = g
        y0 = [2.0 / (g + 1.0), (g + 1.0) / (g - 1.0), 2.0 / (g + 1.0)]
        sol = solve_ivp(_rhs, (1.0, eta_min), y0, args=(g,), method="LSODA",
                        rtol=1e-11, atol=1e-14, dense_output=True)
        if not sol.success:
            raise RuntimeError(sol.message)
        self._sol = sol
        # energy integral on a fine grid, log-spaced towards the centre
        eta = np.concatenate([np.geomspace(eta_min, 0.5, 4000), np.linspace(0.5, 1.0, 4001)[1:]])
        phi, psi, pi_ = sol.sol(eta)
        f = (0.5 * psi * phi ** 2 + pi_ / (g - 1.0)) * eta ** 2
        integral = np.trapezoid(f, eta)
        self.energy_integral = integral
        self.xi0 = (25.0 / (16.0 * math.pi * integral)) ** 0.2

    def shock_radius(self, t, E=1.0, rho0=1.0):
        return self.xi0 * (E * t * t / rho0) ** 0.2

    def profile(self, r, t, E=1.0, rho0=1.0):
        """rho, radial velocity, P at radii r and time t."""
        r = np.atleast_1d(np.asarray(r, dtype=np.float64))
        R = self.shock_radius(t, E, rho0)
        Rdot = 0.4 * R / t
        eta = r / R
        rho = np.full_like(r, rho0)
        v = np.zeros_like(r)
        P = np.zeros_like(r)
        inside = (eta < 1.0) & (eta > self._sol.t[-1])
        if inside.any():
            phi, psi, pi_ = self._sol.sol(eta[inside])
            rho[inside] = rho0 * psi
            v[inside] = Rdot * phi
            P[inside] = rho0 * Rdot * Rdot * pi_
        core = eta <= self._sol.t[-1]
        if core.any():
            phi, psi, pi_ = self._sol.sol(self._sol.t[-1])
            rho[core] = rho0 * psi
            v[core] = 0.0
            P[core] = rho0 * Rdot * Rdot * pi_
        return rho, v, P
