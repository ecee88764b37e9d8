"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated by the method's accuracy target): h and rho to 1e-5
relative, Omega to 1e-5 relative, accelerations, du/dt and div v to 2e-4 of
the per-field max norm; neighbour sets bit-exact except pairs within 1e-6 h
of the support radius (those depend on the last rounding of r)."""
import numpy as np
import pytest

import oracle
from helpers import gpu_evaluate, norm_err, oracle_params, oracle_sampled, rel_max, to_input_order
from paper_2511_11425_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_H = 1e-5
TOL_F = 2e-4


@pytest.fixture(scope="module")
def sph():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2511_11425_gb300 as m
    m.lib()
    return m


def _full_parity(prob, g, fields_only=False):
    p = oracle_params(prob)
    d = oracle.density_h(p, prob.pos, prob.m, prob.h0)
    assert d["failed"] == 0
    f = oracle.forces(p, prob.pos, prob.vel, prob.m, d["h"], d["rho"], d["omega"], prob.u)
    errs = {
        "h": rel_max(g["h"], d["h"]),
        "rho": rel_max(g["rho"], d["rho"]),
        "omega": rel_max(g["omega"], d["omega"]),
        "a": norm_err(g["a"], f["a"]),
        "dudt_h": norm_err(g["dudt_h"], f["dudt_h"]),
        "dudt_av": norm_err(g["dudt_av"], f["dudt_av"]) if np.any(f["dudt_av"]) else 0.0,
        "divv": norm_err(g["divv"], f["divv"]),
        "dt": rel_max(g["dt_i"], f["dt"]),
    }
    return errs, d, f


def _assert_errs(errs):
    assert errs["h"] < TOL_H and errs["rho"] < TOL_H and errs["omega"] < TOL_H, errs
    for k in ("a", "dudt_h", "dudt_av", "divv"):
        assert errs[k] < TOL_F, (k, errs)
    assert errs["dt"] < 1e-4, errs


@pytest.mark.parametrize("n,periodic", [(15, (1, 1, 1)), (17, (1, 1, 1)), (13, (0, 0, 0))])
def test_random_box_parity(sph, n, periodic):
    # n^3 particles: 3375 / 4913 / 2197 -> ragged last bucket, 1-2 sort tiles,
    # random velocities (viscosity active), periodic and open boundaries
    prob = inputs.uniform(n=n, seed=100 + n, jitter=0.35, vamp=0.4, periodic=periodic)
    g = gpu_evaluate(prob)
    errs, d, f = _full_parity(prob, g)
    _assert_errs(errs)


@pytest.mark.parametrize("kernel,nngb", [("wc4", 100), ("wc6", 200), ("m4", 32)])
def test_other_kernels_parity(sph, kernel, nngb):
    prob = inputs.uniform(n=14, seed=7, jitter=0.3, vamp=0.3)
    prob.kernel, prob.n_ngb = kernel, nngb
    prob.h0 = prob.h0 * (nngb / 64.0) ** (1 / 3)
    g = gpu_evaluate(prob)
    errs, d, f = _full_parity(prob, g)
    _assert_errs(errs)


def test_sod_initial_evaluation_parity(sph):
    # the full 15,552-particle Sod tube at t = 0 (every particle compared)
    prob = inputs.sod()
    g = gpu_evaluate(prob)
    errs, d, f = _full_parity(prob, g)
    _assert_errs(errs)
    # neighbour counts at slightly different h differ only for particles with
    # a neighbour right at the support radius
    assert np.mean((g["nngb"].astype(np.int64) & 0xffff) != d["nngb"]) < 1e-3


def test_neighbour_sets_bit_exact(sph):
    import torch
    prob = inputs.uniform(n=12, seed=41, jitter=0.35, vamp=0.0)
    p = oracle_params(prob)
    d = oracle.density_h(p, prob.pos, prob.m, prob.h0)
    h32 = d["h"].astype(np.float32)
    parts = sph.Particles.from_problem(prob, "cuda:0")
    ctx = sph.sph_create(sph.Params.for_problem(prob), prob.n)
    cap = 160
    try:
        sph.sph_build_cells(ctx, parts)
        ids_sorted = parts.t["id"].clone()
        hdev = torch.from_numpy(h32[ids_sorted.cpu().numpy()]).to("cuda:0")
        cnt = torch.zeros(prob.n, dtype=torch.int32, device="cuda:0")
        out = torch.full((prob.n * cap,), -1, dtype=torch.int64, device="cuda:0")
        sph.sph_density_at(ctx, parts, hdev, cap, cnt, out)
        cnt = cnt.cpu().numpy()
        out = out.cpu().numpy().reshape(prob.n, cap)
        sid = ids_sorted.cpu().numpy()
    finally:
        sph.sph_destroy(ctx)
    checked = 0
    for k in range(prob.n):
        i = sid[k]
        nb, margin = oracle.neighbours(p, prob.pos, i, float(h32[i]))
        if margin < 1e-6:
            continue  # a pair sits within 1e-6 h of the support radius
        assert cnt[k] == len(nb)
        assert np.array_equal(np.sort(out[k, :cnt[k]]), nb)
        checked += 1
    assert checked > 0.95 * prob.n


def test_sedov_sampled_parity(sph):
    # the 64^3 Sedov blast at t = 0: every particle on the GPU, sampled sinks
    # (clusters round random centres and the blast centre) in the oracle
    prob = inputs.sedov(n=64)
    g = gpu_evaluate(prob)
    rng = np.random.default_rng(5)
    centres = np.concatenate([rng.random((5, 3)), [[0.5, 0.5, 0.5]]])
    sinks = []
    for c in centres:
        dd = prob.pos - c
        dd -= np.round(dd)
        sinks.extend(np.argsort((dd * dd).sum(1))[:24])
    sinks = np.unique(np.array(sinks))
    o = oracle_sampled(prob, oracle_params(prob), sinks)
    assert rel_max(g["h"][sinks], o["h"]) < TOL_H
    assert rel_max(g["rho"][sinks], o["rho"]) < TOL_H
    assert rel_max(g["omega"][sinks], o["omega"]) < TOL_H
    for k, gk in (("a", g["a"]), ("dudt_h", g["dudt_h"]), ("dudt_av", g["dudt_av"]),
                  ("divv", g["divv"])):
        assert norm_err(gk[sinks], o[k]) < TOL_F, k


def test_conservation_on_gpu(sph):
    prob = inputs.uniform(n=16, seed=3, jitter=0.35, vamp=0.5)
    g = gpu_evaluate(prob)
    m = prob.m
    mom = np.abs((m[:, None] * g["a"]).sum(0)) / (m[:, None] * np.abs(g["a"])).sum(0)
    assert np.all(mom < 1e-5)
    work = m * ((prob.vel * g["a"]).sum(1) + g["dudt_h"] + g["dudt_av"])
    assert abs(work.sum()) < 1e-4 * np.abs(m * (prob.vel * g["a"]).sum(1)).sum()
    st = g["stats"]
    assert st["force_pairs"] > 0 and st["density_pairs"] > 0


def test_sod_twenty_steps_track_oracle(sph):
    # t = 0 evaluation + 20 kick-drift-kick steps with a fixed global step on
    # both sides; positions, velocities and u stay within the force tolerance
    prob = inputs.sod()
    p = oracle_params(prob)
    dt = 0.001
    sim = oracle.Simulation(p, prob.pos, prob.vel, prob.m, prob.u, prob.h0)
    for _ in range(20):
        sim.step(dt_fixed=dt)
    s = sph.Simulation(prob)
    try:
        E0 = s.conserved()
        for _ in range(20):
            s.step(dt_fixed=dt)
        E1 = s.conserved()
        g = to_input_order(s.parts.numpy())
    finally:
        s.close()
    L = np.array(prob.box_hi) - np.array(prob.box_lo)
    dx = g["x"] - sim.x
    dx -= L * np.round(dx / L)
    assert np.max(np.abs(dx)) < 1e-6
    assert norm_err(g["v"], sim.v) < TOL_F
    assert norm_err(g["u"], sim.u) < 1e-5
    # momentum stays zero, total energy drifts like the oracle's
    assert abs(E1[1]) < 1e-6 * E1[0] and abs(E1[2]) < 1e-9 and abs(E1[3]) < 1e-9
    Eg = (E1[7] + E1[8] - E0[7] - E0[8]) / (E0[7] + E0[8])
    assert abs(Eg) < 1e-3


@pytest.mark.parametrize("memory", ["pinned", "pageable", "mixed"])
def test_step_host_matches_device_step(sph, memory):
    """sph_step_host moves pinned arrays with its copy kernel and the others
    with copy-engine transfers; 'mixed' has pageable arrays and a pinned array
    whose start is not 16-byte aligned (byte-wise copy) beside pinned ones."""
    import torch
    prob = inputs.uniform(n=10, seed=8, jitter=0.3, vamp=0.2)
    dev = sph.Simulation(prob)
    try:
        dt_dev = dev.step()
        gd = to_input_order(dev.parts.numpy())
    finally:
        dev.close()
    host = sph.Particles.from_problem(prob, "cpu", pin=memory != "pageable")
    if memory == "mixed":
        for f in ("u", "v1", "rho", "iters"):
            host.t[f] = host.t[f].clone()      # pageable copies
        shifted = torch.zeros(prob.n + 1, dtype=torch.float32, pin_memory=True)[1:]
        shifted.copy_(host.t["h"])
        host.t["h"] = shifted                  # pinned, 4 bytes past a 16-byte boundary
        assert host.t["h"].data_ptr() % 16 == 4 and host.t["h"].is_pinned()
    ctx = sph.sph_create(sph.Params.for_problem(prob), prob.n)
    try:
        dt_h, hb, db = sph.sph_step_host(ctx, host)
    finally:
        sph.sph_destroy(ctx)
    gh = to_input_order(host.numpy())
    assert abs(dt_h - dt_dev) < 1e-6 * dt_dev
    assert hb == 92 * prob.n and db == 111 * prob.n   # step inputs in, every array out
    assert norm_err(gh["a"], gd["a"]) < 1e-5
    assert np.max(np.abs(gh["x"] - gd["x"])) < 1e-9


def test_conserved_reduction_matches_numpy(sph):
    prob = inputs.uniform(n=9, seed=4, vamp=0.3)
    s = sph.Simulation(prob)
    try:
        out = np.array(s.conserved())
        out2 = np.array(s.conserved())
    finally:
        s.close()
    want = oracle.conserved(prob.pos, prob.vel, prob.m.astype(np.float32).astype(np.float64),
                            prob.u)
    assert np.allclose(out, want, rtol=1e-12, atol=1e-15)
    assert np.array_equal(out, out2)  # fixed-order reduction


def test_isentropic_mode_tracks_oracle(sph):
    prob = inputs.uniform(n=10, seed=12, jitter=0.3, vamp=0.3)
    p = oracle_params(prob)
    sim = oracle.Simulation(p, prob.pos, prob.vel, prob.m, prob.u, prob.h0, energy="isentropic")
    prm = sph.Params.for_problem(prob, energy="isentropic")
    s = sph.Simulation(prob, prm)
    try:
        for _ in range(3):
            sim.step(dt_fixed=2e-3)
            s.step(dt_fixed=2e-3)
        g = to_input_order(s.parts.numpy())
    finally:
        s.close()
    assert norm_err(g["u"], sim.u) < 1e-5
    assert norm_err(g["v"], sim.v) < TOL_F


def test_edge_cases_and_errors(sph):
    import torch
    prm = sph.Params()
    # empty input: every call succeeds and does nothing
    empty = sph.Particles(0, "cuda:0")
    ctx = sph.sph_create(prm, 0)
    try:
        sph.sph_build_cells(ctx, empty)
        sph.sph_density_h(ctx, empty)
        sph.sph_forces(ctx, empty)
        sph.sph_kdk_step(ctx, empty, 1e-3)
    finally:
        sph.sph_destroy(ctx)
    # a single ragged bucket (n < 32), open box, small neighbour number
    prob = inputs.uniform(n=3, seed=2, jitter=0.2, periodic=(0, 0, 0))
    prob.n_ngb = 20.0
    g = gpu_evaluate(prob)
    errs, d, f = _full_parity(prob, g)
    _assert_errs(errs)
    # out-of-order calls and bad sizes are reported, not crashed on
    prob = inputs.uniform(n=4, seed=2)
    parts = sph.Particles.from_problem(prob, "cuda:0")
    ctx = sph.sph_create(sph.Params.for_problem(prob), prob.n - 1)
    try:
        with pytest.raises(sph.SphError) as e:
            sph.sph_build_cells(ctx, parts)
        assert e.value.code == 1
    finally:
        sph.sph_destroy(ctx)
    ctx = sph.sph_create(sph.Params.for_problem(prob), prob.n)
    try:
        with pytest.raises(sph.SphError) as e:
            sph.sph_forces(ctx, parts)
        assert e.value.code == 7
        parts.t["x0"][5] = float("nan")
        with pytest.raises(sph.SphError) as e:
            sph.sph_build_cells(ctx, parts)
        assert e.value.code == 5
    finally:
        sph.sph_destroy(ctx)
    torch.cuda.synchronize()
