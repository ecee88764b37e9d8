"""Hierarchical power-of-two time steps (Sec. 2.3.6) on the GPU against the
oracle's integrator of the same scheme (oracle.RungSimulation), through the
C ABI (sph_step_rungs): a Sedov blast on 12^3 particles whose hot centre
sits four rungs above the cold gas, two global steps of 16 substeps.  The
rungs must agree exactly (the test first checks that no rung decision of
the oracle lies within 2e-3 of a power-of-two boundary in log2 units, where
FP32 and FP64 time-step limits could round to different rungs: the limits
of the two agree to about 1e-5 relative, 1.4e-5 in log2 units); positions, velocities and
internal energies within the tolerances of the global-step tracking test."""
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


def _compare(sph, prob, dt0, R, nglobal, fastgas=True):
    p = oracle_params(prob)
    o = oracle.RungSimulation(p, prob.pos, prob.vel, prob.m, prob.u, prob.h0, max_rung=R)
    for _ in range(nglobal):
        o.global_step(dt0)
    dist = min(float(np.min(np.abs(r - np.round(r)))) for _, _, r in o.log if len(r))
    assert dist > 2e-3, dist
    sim = sph.Simulation(prob)
    try:
        sph.sph_set_fastgas(sim.ctx, fastgas)
        for _ in range(nglobal):
            sph.sph_step_rungs(sim.ctx, sim.parts, dt0, R)
        g = sim.parts.numpy()
        rungs = sph.sph_get_rungs(sim.ctx, prob.n)
    finally:
        sim.close()
    order = np.argsort(g["id"], kind="stable")
    rungs = rungs[order]
    g = to_input_order(g)
    L = np.array(prob.box_hi) - np.array(prob.box_lo)
    dx = g["x"] - o.x
    dx -= L * np.round(dx / L)
    errs = {"x": float(np.max(np.abs(dx))), "v": norm_err(g["v"], o.v),
            "u": norm_err(g["u"], o.u)}
    print("rungs", np.bincount(rungs, minlength=R + 1), {k: "%.2g" % v for k, v in errs.items()})
    return errs, rungs, o


@pytest.mark.parametrize("fastgas", [True, False])
def test_rungs_track_oracle_sedov(sph, fastgas):
    prob = inputs.sedov(n=12)
    errs, rungs, o = _compare(sph, prob, 0.018, 4, 2, fastgas)
    assert np.array_equal(rungs, o.rung)
    assert len(np.unique(rungs)) >= 3                  # a real hierarchy
    assert errs["x"] < 1e-6 and errs["v"] < 2e-4 and errs["u"] < 1e-5


def test_rungs_arguments(sph):
    prob = inputs.uniform(n=6, seed=3)
    sim = sph.Simulation(prob)
    try:
        with pytest.raises(sph.SphError) as e:
            sph.sph_step_rungs(sim.ctx, sim.parts, -1.0, 2)
        assert e.value.code == 1
        sph.sph_step_rungs(sim.ctx, sim.parts, 1e-3, 2)
        with pytest.raises(sph.SphError) as e:
            sph.sph_step_rungs(sim.ctx, sim.parts, 1e-3, 3)   # one max_rung per run
        assert e.value.code == 7
    finally:
        sim.close()
    sim = sph.Simulation(prob)
    try:
        sim.step(1e-3)
        with pytest.raises(sph.SphError) as e:                 # begun with global steps
            sph.sph_step_rungs(sim.ctx, sim.parts, 1e-3, 2)
        assert e.value.code == 7
    finally:
        sim.close()


def _rung_run(sph, prob, dt0, R, nglobal, fastgas):
    import time
    import torch
    sim = sph.Simulation(prob)
    try:
        sph.sph_set_fastgas(sim.ctx, fastgas)
        sph.sph_step_rungs(sim.ctx, sim.parts, dt0, R)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(nglobal - 1):
            sph.sph_step_rungs(sim.ctx, sim.parts, dt0, R)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        g = sim.parts.numpy()
        rungs = sph.sph_get_rungs(sim.ctx, prob.n)[np.argsort(g["id"], kind="stable")]
        return to_input_order(g), rungs, secs
    finally:
        sim.close()


def test_fastgas_matches_full_substeps(sph):
    # a Sedov blast on 32^3 particles with six rungs: most substeps activate
    # only the hot centre.  FastGas solves the marked neighbourhoods only;
    # the active particles see the same partners with the same densities (to
    # the Newton tolerance: the marked particles start from older seeds), so
    # the state after the global steps is the one of full substeps
    prob = inputs.sedov(n=32)
    R = 6
    sim = sph.Simulation(prob)
    try:
        sph.sph_build_cells(sim.ctx, sim.parts)
        sph.sph_density_h(sim.ctx, sim.parts)
        sph.sph_forces(sim.ctx, sim.parts)
        dt_min = float(np.min(sim.parts.numpy()["dt_i"]))
    finally:
        sim.close()
    dt0 = 2 ** R * dt_min * 0.9          # the hottest particles on the top rung
    full, r_full, t_full = _rung_run(sph, prob, dt0, R, 3, False)
    fast, r_fast, t_fast = _rung_run(sph, prob, dt0, R, 3, True)
    print("rungs", np.bincount(r_full, minlength=R + 1), "full %.3fs fastgas %.3fs" %
          (t_full, t_fast))
    assert len(np.unique(r_full)) >= 4
    assert np.mean(r_full != r_fast) < 1e-3
    L = np.array(prob.box_hi) - np.array(prob.box_lo)
    dx = fast["x"] - full["x"]
    dx -= L * np.round(dx / L)
    assert np.max(np.abs(dx)) < 1e-7
    assert norm_err(fast["v"], full["v"]) < 2e-4
    assert norm_err(fast["u"], full["u"]) < 1e-5
