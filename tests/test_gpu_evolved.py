"""The evolved-density variant (Sec. 2.3.3: rho integrated with the mass
conservation equation, the density pass still giving h and Omega) on the
GPU against the oracle's integrator of the same variant (oracle.Simulation,
density='evolved'), through the C ABI: a compressive flow in a periodic box
and the Sod tube, stepped with a fixed global step."""
import numpy as np
import pytest

import oracle
from helpers import norm_err, oracle_params, to_input_order
from paper_2511_11425_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2511_11425_gb300 as m
    m.lib()
    return m


def _track(sph, prob, dt, steps):
    p = oracle_params(prob)
    osim = oracle.Simulation(p, prob.pos, prob.vel, prob.m, prob.u, prob.h0, density="evolved")
    for _ in range(steps):
        osim.step(dt_fixed=dt)
    s = sph.Simulation(prob, sph.Params.for_problem(prob, density="evolved"))
    try:
        for _ in range(steps):
            s.step(dt_fixed=dt)
        g = to_input_order(s.parts.numpy())
    finally:
        s.close()
    L = np.array(prob.box_hi) - np.array(prob.box_lo)
    dx = g["x"] - osim.x
    dx -= L * np.round(dx / L)
    errs = {"x": float(np.max(np.abs(dx))), "v": norm_err(g["v"], osim.v),
            "u": norm_err(g["u"], osim.u),
            "rho": float(np.max(np.abs(g["rho"] - osim.rho) / osim.rho)),
            "h": float(np.max(np.abs(g["h"] - osim.h) / osim.h))}
    print(prob.name, {k: "%.2g" % v for k, v in errs.items()})
    return errs, g, osim


def test_evolved_density_tracks_oracle_compressive_flow(sph):
    prob = inputs.uniform(n=12, seed=51, jitter=0.25, vamp=0.0)
    prob.vel[:, 0] = 0.3 * np.sin(2 * np.pi * prob.pos[:, 0])
    prob.vel[:, 1] = 0.1 * np.cos(2 * np.pi * prob.pos[:, 2])
    errs, g, osim = _track(sph, prob, 2e-3, 8)
    assert errs["x"] < 1e-6 and errs["v"] < 2e-4 and errs["u"] < 1e-5
    assert errs["rho"] < 1e-5
    # the evolved density is not the kernel sum any more (it is state)
    assert np.max(np.abs(osim.rho - osim.last["rho"]) / osim.rho) > 1e-5


def test_evolved_density_tracks_oracle_sod(sph):
    prob = inputs.sod()
    errs, g, osim = _track(sph, prob, 1e-3, 10)
    assert errs["x"] < 1e-6 and errs["v"] < 2e-4 and errs["u"] < 1e-5
    assert errs["rho"] < 1e-5


def test_evolved_density_mode_arguments(sph):
    with pytest.raises(sph.SphError) as e:
        sph.sph_create(sph.Params(density="evolved", energy="isentropic"), 10)
    assert e.value.code == 1
    # a step must precede the recording of a step (the evolved density starts
    # from the first kernel sum)
    import torch
    prob = inputs.uniform(n=6, seed=52)
    sim = sph.Simulation(prob, sph.Params.for_problem(prob, density="evolved"))
    try:
        s = torch.cuda.Stream()
        with pytest.raises(sph.SphError) as e:
            sph.sph_graph_capture(sim.ctx, sim.parts, 1e-3, s)
        assert e.value.code == 7
        sph.sph_step(sim.ctx, sim.parts, 1e-3, s)
        sph.sph_graph_capture(sim.ctx, sim.parts, 1e-3, s)
        sph.sph_graph_launch(sim.ctx, s)
    finally:
        sim.close()
