"""Shared helpers for the GPU tests: run the C-ABI path on a Problem and map
results back to input order; run the FP64 oracle on the same inputs."""
import numpy as np

import oracle


def oracle_params(prob, **kw):
    d = dict(kernel=prob.kernel, n_ngb=prob.n_ngb, gamma=prob.gamma, alpha=prob.alpha,
             beta=prob.beta, box_lo=prob.box_lo, box_hi=prob.box_hi, periodic=prob.periodic)
    d.update(kw)
    return oracle.Params(**d)


def to_input_order(g):
    """Arrays of a Particles.numpy() dict, re-indexed by particle id."""
    order = np.argsort(g["id"], kind="stable")
    out = {k: v[order] for k, v in g.items()}
    out["a"] = np.stack([out["a0"], out["a1"], out["a2"]], 1)
    out["x"] = np.stack([out["x0"], out["x1"], out["x2"]], 1)
    out["v"] = np.stack([out["v0"], out["v1"], out["v2"]], 1)
    return out


def gpu_evaluate(prob, params=None, device="cuda:0"):
    """build_cells + density_h + forces on the GPU; results in input order."""
    import paper_2511_11425_gb300 as sph
    prm = params or sph.Params.for_problem(prob)
    parts = sph.Particles.from_problem(prob, device)
    ctx = sph.sph_create(prm, prob.n)
    try:
        sph.sph_build_cells(ctx, parts)
        sph.sph_density_h(ctx, parts)
        sph.sph_forces(ctx, parts)
        stats = sph.sph_get_stats(ctx)
        g = to_input_order(parts.numpy())
    finally:
        sph.sph_destroy(ctx)
    g["stats"] = stats
    return g


def rel_max(gpu, ref):
    return float(np.max(np.abs(gpu - ref) / np.abs(ref)))


def norm_err(gpu, ref):
    """max_i |gpu - ref| / max_i |ref| (per-field max-norm error)."""
    return float(np.max(np.abs(gpu - ref)) / max(np.max(np.abs(ref)), 1e-300))


def oracle_neighbourhood(prob, sinks, radius):
    """Indices within `radius` of any sink (minimum image on periodic axes)."""
    keep = np.zeros(prob.n, dtype=bool)
    L = np.array(prob.box_hi) - np.array(prob.box_lo)
    per = np.array(prob.periodic, dtype=bool)
    for s in sinks:
        d = prob.pos - prob.pos[s]
        d[:, per] -= L[per] * np.round(d[:, per] / L[per])
        keep |= (d * d).sum(1) < radius * radius
    return np.nonzero(keep)[0]


def oracle_sampled(prob, p, sinks, hood_factor=2.2, radius=None):
    """Oracle density + forces for the sinks only, exact for them.

    Density (h, rho, Omega) is solved by brute force over all N for every
    particle within hood_factor * h_seed_max of a sink, which contains every
    particle that can interact with a sink; forces are then evaluated for the
    sinks with those values (particles outside the neighbourhood get h = 0,
    so they cannot enter a sink's sums).
    """
    sinks = np.asarray(sinks)
    R = radius if radius is not None else hood_factor * float(np.max(prob.h0))
    hood = oracle_neighbourhood(prob, sinks, R)
    d = oracle.density_h(p, prob.pos, prob.m, prob.h0, hood)
    assert d["failed"] == 0
    h = np.zeros(prob.n)
    rho = np.ones(prob.n)
    om = np.ones(prob.n)
    h[hood] = d["h"]
    rho[hood] = d["rho"]
    om[hood] = d["omega"]
    # every particle within max(h) of a sink must be inside the neighbourhood
    assert float(np.max(h)) * 1.05 + float(np.max(h[sinks])) < R
    f = oracle.forces(p, prob.pos, prob.vel, prob.m, h, rho, om, prob.u, sinks)
    return {"h": h[sinks], "rho": rho[sinks], "omega": om[sinks], **f}


def motion_err(xa, xb, prob):
    """max |xa - xb| over the largest displacement of xb from the initial
    positions of prob (minimum image on periodic axes).  Two GPU runs differ
    by the reassociation of float atomics in the force sums, so their
    positions agree relative to how far the particles moved, not absolutely."""
    L = np.array(prob.box_hi) - np.array(prob.box_lo)
    per = np.array(prob.periodic) > 0

    def wrap(d):
        return d - np.where(per, L * np.round(d / L), 0.0)
    mv = np.max(np.abs(wrap(xb - prob.pos)))
    return np.max(np.abs(wrap(xa - xb))) / max(mv, 1e-300)
