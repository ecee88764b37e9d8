"""Batched form and captured steps.

* A batch context steps independent problems of uneven sizes, boxes,
  periodicities and gases in one launch per phase; every instance must
  evolve exactly as when it is stepped alone (same pairs, same step sizes,
  fields within the force tolerance), and its conserved totals must be its
  own.
* A step captured once as a CUDA graph and replayed must reproduce plain
  sph_step calls."""
import numpy as np
import pytest

from helpers import motion_err, norm_err, to_input_order
from paper_2511_11425_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2511_11425_gb300 as m
    m.lib()
    return m


def _problems():
    return [inputs.sod(length_cells=24, seed=1),
            inputs.sedov(n=14, seed=2),
            inputs.uniform(n=9, seed=3, vamp=0.3, periodic=(0, 0, 0)),
            inputs.uniform(n=7, seed=4, vamp=0.2, jitter=0.3)]


def test_batch_steps_like_separate_problems(sph):
    probs = _problems()
    params = [sph.Params.for_problem(p) for p in probs]
    parts, offs = sph.Particles.from_problems(probs, "cuda:0")
    assert list(offs) == list(np.cumsum([0] + [p.n for p in probs]))
    ctx = sph.sph_batch_create(params, offs)
    try:
        for _ in range(3):
            sph.sph_step(ctx, parts)
        dts = sph.sph_batch_get_dt(ctx, len(probs))
        tot = np.array(sph.sph_reduce_conserved(ctx, parts)).reshape(len(probs), 9)
        st = sph.sph_get_stats(ctx)
        g = to_input_order(parts.numpy())
    finally:
        sph.sph_destroy(ctx)
    pairs = 0
    for k, p in enumerate(probs):
        s = sph.Simulation(p)
        try:
            for _ in range(3):
                dt = s.step()
            pairs += sph.sph_get_stats(s.ctx)["force_pairs"]
            one = to_input_order(s.parts.numpy())
            tot1 = np.array(s.conserved())
        finally:
            s.close()
        sl = slice(offs[k], offs[k + 1])
        assert abs(dts[k] - dt) <= 1e-5 * dt, (k, dts[k], dt)
        L = np.array(p.box_hi) - np.array(p.box_lo)
        assert motion_err(g["x"][sl], one["x"], p) < 1e-5, k
        assert norm_err(g["a"][sl], one["a"]) < 1e-5, k
        assert np.max(np.abs(g["h"][sl] - one["h"]) / one["h"]) < 1e-5, k
        # mass and energies agree closely; momentum and angular momentum are
        # round-off zeros, compared on the momentum scale sqrt(2 M E_kin)
        assert np.allclose(tot[k][[0, 7, 8]], tot1[[0, 7, 8]], rtol=1e-6), k
        pscale = np.sqrt(2.0 * tot1[0] * max(tot1[7], 1e-30)) * max(1.0, float(np.max(L)))
        assert np.max(np.abs(tot[k][1:7] - tot1[1:7])) < 1e-6 * pscale + 1e-14, k
    # the last step's pair count is the sum over instances (pairs right at a
    # support radius may flip with the last rounding of a position)
    assert abs(st["force_pairs"] - pairs) <= 1e-4 * pairs


def test_graph_replay_matches_plain_steps(sph):
    import torch
    prob = inputs.uniform(n=16, seed=9, vamp=0.3, jitter=0.3)
    stream = torch.cuda.Stream()
    a = sph.Simulation(prob)
    b = sph.Simulation(prob)
    try:
        with torch.cuda.stream(stream):
            dta = [sph.sph_step(a.ctx, a.parts, 0.0, stream) for _ in range(4)]
            dtb = [sph.sph_step(b.ctx, b.parts, 0.0, stream)]
            sph.sph_graph_capture(b.ctx, b.parts, 0.0, stream)
            dtb += [sph.sph_graph_launch(b.ctx, stream) for _ in range(3)]
        stream.synchronize()
        ga = to_input_order(a.parts.numpy())
        gb = to_input_order(b.parts.numpy())
        st = sph.sph_get_stats(b.ctx)
        launches = st["launches"]
        # the replay carries the totals of the stepped state and phase times
        assert sph.sph_graph_totals(b.ctx) == sph.sph_reduce_conserved(b.ctx, b.parts)
        assert st["ms_density_kernel"] > 0 and st["ms_force_kernel"] > 0
    finally:
        a.close()
        b.close()
    assert np.allclose(dta, dtb, rtol=1e-5)
    assert motion_err(gb["x"], ga["x"], prob) < 1e-5
    assert norm_err(gb["v"], ga["v"]) < 1e-5
    assert norm_err(gb["a"], ga["a"]) < 1e-5
    assert launches > 0


def test_step_host_replays_captured_step(sph):
    """sph_step_host after sph_step_host_capture replays the recorded step on
    the context's device buffers: same states as plain device steps, only the
    step's inputs copied in, every array copied out."""
    import torch
    prob = inputs.uniform(n=14, seed=12, vamp=0.3, jitter=0.3)
    stream = torch.cuda.Stream()
    a = sph.Simulation(prob)
    host = sph.Particles.from_problem(prob, "cpu", pin=True)
    ctx = sph.sph_create(sph.Params.for_problem(prob), prob.n)
    try:
        with torch.cuda.stream(stream):
            dta = [sph.sph_step(a.ctx, a.parts, 0.0, stream) for _ in range(4)]
        stream.synchronize()
        ga = to_input_order(a.parts.numpy())
        dtb = [sph.sph_step_host(ctx, host, 0.0, stream)[0]]
        with pytest.raises(sph.SphError):
            sph.sph_graph_totals(ctx)                     # nothing replayed yet
        sph.sph_step_host_capture(ctx, host, 0.0, stream)
        for _ in range(3):
            dt, hb, db = sph.sph_step_host(ctx, host, 0.0, stream)
            dtb.append(dt)
        totals = sph.sph_graph_totals(ctx)                # set by a replay
    finally:
        a.close()
        sph.sph_destroy(ctx)
    gb = to_input_order(host.numpy())
    assert len(totals) == 9
    assert np.allclose(dta, dtb, rtol=1e-5)
    assert motion_err(gb["x"], ga["x"], prob) < 1e-5
    assert norm_err(gb["v"], ga["v"]) < 1e-5
    assert norm_err(gb["a"], ga["a"]) < 1e-5
    # outputs copied back while the replay finishes (density and force
    # outputs) arrive complete, like the ones copied after it
    for f in ("rho", "omega", "h", "u", "dt_i"):
        assert norm_err(gb[f], ga[f]) < 1e-5, f
    assert norm_err(gb["divv"], ga["divv"]) < 1e-3
    assert np.mean(gb["nngb"] != ga["nngb"]) < 1e-2 and np.all(gb["iters"] >= 1)
    # inputs only in (x, v, u: 7 x 8 B; m, h, a, du/dt: 7 x 4 B; id 8 B),
    # everything out (111 B per particle)
    assert hb == 92 * prob.n and db == 111 * prob.n


def test_step_host_isentropic_replay_matches_device_steps(sph):
    """In the entropy-conserving mode rho is a step input (read before the
    density pass) and u is first read after it (copied in beside the step):
    host-buffer steps, plain and replayed, follow plain device steps."""
    import torch
    prob = inputs.uniform(n=12, seed=21, vamp=0.3, jitter=0.3)
    prm = sph.Params.for_problem(prob, energy="isentropic", resort_period=2)
    stream = torch.cuda.Stream()
    a = sph.Simulation(prob, prm)
    host = sph.Particles.from_problem(prob, "cpu", pin=True)
    ctx = sph.sph_create(prm, prob.n)
    try:
        with torch.cuda.stream(stream):
            dta = [sph.sph_step(a.ctx, a.parts, 0.0, stream) for _ in range(5)]
        stream.synchronize()
        ga = to_input_order(a.parts.numpy())
        dtb = [sph.sph_step_host(ctx, host, 0.0, stream)[0]]
        sph.sph_step_host_capture(ctx, host, 0.0, stream)
        in_bytes, out_bytes = [], []
        for _ in range(4):                                # re-sorting and refitting replays
            dt, hb, db = sph.sph_step_host(ctx, host, 0.0, stream)
            dtb.append(dt)
            in_bytes.append(hb)
            out_bytes.append(db)
    finally:
        a.close()
        sph.sph_destroy(ctx)
    gb = to_input_order(host.numpy())
    assert np.allclose(dta, dtb, rtol=1e-5)
    assert motion_err(gb["x"], ga["x"], prob) < 1e-5
    for f in ("v", "a", "u", "rho", "h"):
        assert norm_err(gb[f], ga[f]) < 1e-5, f
    # a refitting replay reads no id (8 B per particle not copied in; rho
    # is an input in this mode) and leaves m and id on the host as they were
    # (12 B per particle not copied back); the ids still order the particles
    assert sorted(set(in_bytes)) == [88 * prob.n, 96 * prob.n]
    assert sorted(set(out_bytes)) == [99 * prob.n, 111 * prob.n]
    assert np.array_equal(gb["m"], ga["m"]) and np.array_equal(np.sort(gb["id"]), np.arange(prob.n))


def test_replayed_rewalk_rounds_match_plain_steps(sph):
    """Seeding every density pass 20 % below the converged h (the seed is
    the h array the step starts from) puts the root beyond the lists'
    10 % coverage, so the re-walk rounds do work, in plain steps and inside
    replayed graphs alike.  Replays give the plain steps' states and report
    their re-walks."""
    import torch
    prob = inputs.uniform(n=12, seed=33, vamp=0.3, jitter=0.3)
    prm = sph.Params.for_problem(prob)
    stream = torch.cuda.Stream()
    a = sph.Simulation(prob, prm)
    b = sph.Simulation(prob, prm)
    try:
        with torch.cuda.stream(stream):
            dta, dtb, relists_a, relists_b = [], [], [], []
            for k in range(4):
                a.parts.t["h"].mul_(0.8)
                dta.append(sph.sph_step(a.ctx, a.parts, 0.0, stream))
                relists_a.append(sph.sph_get_stats(a.ctx)["relists"])
            b.parts.t["h"].mul_(0.8)
            dtb.append(sph.sph_step(b.ctx, b.parts, 0.0, stream))
            sph.sph_graph_capture(b.ctx, b.parts, 0.0, stream)
            for _ in range(3):
                b.parts.t["h"].mul_(0.8)
                dtb.append(sph.sph_graph_launch(b.ctx, stream))
                relists_b.append(sph.sph_get_stats(b.ctx)["relists"])
        stream.synchronize()
        ga = to_input_order(a.parts.numpy())
        gb = to_input_order(b.parts.numpy())
    finally:
        a.close()
        b.close()
    assert min(relists_a) > 0 and min(relists_b) > 0   # the rounds ran inside the replays
    assert np.allclose(dta, dtb, rtol=1e-5)
    assert motion_err(gb["x"], ga["x"], prob) < 1e-5
    for f in ("h", "rho", "omega", "v", "a"):
        assert norm_err(gb[f], ga[f]) < 1e-5, f


def test_batch_simulation_graph_matches_plain_batch(sph):
    """BatchSimulation replaying a captured step advances every instance like
    plain batch steps (same step sizes, same state)."""
    import torch
    probs = _problems()
    stream = torch.cuda.Stream()
    a = sph.BatchSimulation(probs)
    b = sph.BatchSimulation(probs)
    try:
        with torch.cuda.stream(stream):
            da = [a.step(0.0, stream) for _ in range(3)]
            db = [b.step(0.0, stream)]
            b.capture(stream)
            db += [b.step() for _ in range(2)]
        stream.synchronize()
        ga = to_input_order(a.parts.numpy())
        gb = to_input_order(b.parts.numpy())
        ca = np.array(a.conserved()).reshape(len(probs), 9)
        cb = np.array(b.conserved()).reshape(len(probs), 9)
    finally:
        a.close()
        b.close()
    assert np.allclose(np.array(da), np.array(db), rtol=1e-5)
    assert np.allclose(a.t, b.t, rtol=1e-5)
    for k, p in enumerate(probs):
        sl = slice(a.offsets[k], a.offsets[k + 1])
        assert motion_err(gb["x"][sl], ga["x"][sl], p) < 1e-5, k
    assert norm_err(gb["a"], ga["a"]) < 1e-5
    assert np.allclose(ca[:, [0, 7, 8]], cb[:, [0, 7, 8]], rtol=1e-6)


def test_resort_period_refits_between_sorts(sph):
    """With resort_period 4, three of every four steps keep the bucket layout
    and only refit its bounds: fewer kernels per step, the same motion (up to
    summation order), in plain steps and in graph replays."""
    import torch
    prob = inputs.uniform(n=16, seed=13, vamp=0.4, jitter=0.3)
    stream = torch.cuda.Stream()
    runs = {}
    for name, period, graph in (("sorted", 1, False), ("refit", 4, False),
                                ("refit_graph", 4, True)):
        s = sph.Simulation(prob, sph.Params.for_problem(prob, resort_period=period))
        try:
            with torch.cuda.stream(stream):
                launches = []
                if graph:
                    sph.sph_step(s.ctx, s.parts, 0.0, stream)
                    sph.sph_graph_capture(s.ctx, s.parts, 0.0, stream)
                for k in range(8 if not graph else 7):
                    l0 = sph.sph_get_stats(s.ctx)["launches"]
                    if graph:
                        sph.sph_graph_launch(s.ctx, stream)
                    else:
                        sph.sph_step(s.ctx, s.parts, 0.0, stream)
                    launches.append(sph.sph_get_stats(s.ctx)["launches"] - l0)
            stream.synchronize()
            runs[name] = (to_input_order(s.parts.numpy()), launches)
        finally:
            s.close()
    ref, lref = runs["sorted"]
    for name in ("refit", "refit_graph"):
        g, ln = runs[name]
        assert motion_err(g["x"], ref["x"], prob) < 1e-5, name
        assert norm_err(g["a"], ref["a"]) < 1e-5, name
        assert min(ln) < min(lref), name      # refit steps launch fewer kernels
    assert runs["refit"][1][0] == lref[0]     # the first step re-sorts
