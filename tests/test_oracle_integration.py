"""End-to-end pin of the oracle: a Sod tube (Sec. 3.2 initial states, half the
resolution of the parity case) integrated with the global-step
kick-drift-kick scheme (Sec. 2.3.6) to t = 0.1, compared with the exact
Riemann solution, plus total-energy conservation of the PdV form."""
import numpy as np
import pytest

import oracle
from oracle import riemann
from paper_2511_11425_gb300 import inputs


@pytest.fixture(scope="module")
def sod_run():
    pr = inputs.sod(length_cells=48)
    p = oracle.Params(gamma=pr.gamma, alpha=pr.alpha, beta=pr.beta, box_lo=pr.box_lo,
                      box_hi=pr.box_hi, periodic=pr.periodic)
    sim = oracle.Simulation(p, pr.pos, pr.vel, pr.m, pr.u, pr.h0)
    E = []
    while sim.t < 0.1:
        dt = sim.step()
        v_i = sim.v - 0.5 * dt * sim.a
        u_i = sim.u - 0.5 * dt * sim.udot
        E.append(float((sim.m * (0.5 * (v_i ** 2).sum(1) + u_i)).sum()))
    return pr, sim, np.array(E)


def test_sod_energy_and_momentum(sod_run):
    pr, sim, E = sod_run
    assert np.max(np.abs(E - E[0])) < 1e-4 * E[0]
    mom = (sim.m[:, None] * sim.v).sum(0)
    assert np.max(np.abs(mom)) < 1e-12


def test_sod_matches_riemann_solution(sod_run):
    pr, sim, E = sod_run
    x = sim.x[:, 0]
    rho = sim.last["rho"]
    P = (pr.gamma - 1) * rho * sim.u
    bins = np.linspace(-0.3, 0.3, 31)
    c = 0.5 * (bins[1:] + bins[:-1])
    idx = np.digitize(x, bins) - 1
    ok = (idx >= 0) & (idx < 30)

    def prof(q):
        return np.array([q[ok & (idx == k)].mean() for k in range(30)])

    ra, ua, pa = riemann.sample(c / sim.t, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    # SPH smooths the jumps over ~h; the L1 norms below sit ~1.5x above the
    # measured 0.040 / 0.104 / 0.043 of this resolution
    assert np.mean(np.abs(prof(rho) - ra)) < 0.06
    assert np.mean(np.abs(prof(sim.v[:, 0]) - ua)) < 0.15
    assert np.mean(np.abs(prof(P) - pa)) < 0.065
