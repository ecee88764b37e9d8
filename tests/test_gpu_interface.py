"""The interface correction (Sec. 2.3.4) on the GPU against the oracle:
the kernel imbalance from the density pass, the exp(-I^2)-weighted averages
of T and P in the correction pass and the corrected density from each
material's ideal-gas EOS feed the force pass; the forces must match the
oracle's forces evaluated at the oracle's corrected density, on two
materials in pressure and temperature equilibrium across a density jump."""
import numpy as np
import pytest

import oracle
from helpers import norm_err, oracle_params, rel_max, to_input_order
from test_oracle_interface import slab_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2511_11425_gb300 as m
    m.lib()
    return m


def _gpu(sph, prob, ic):
    prm = sph.Params.for_problem(prob, interface_correction=ic, r_gas=prob.extra["r_gas"])
    parts = sph.Particles.from_problem(prob, "cuda:0")
    ctx = sph.sph_create(prm, prob.n)
    try:
        sph.sph_build_cells(ctx, parts)
        sph.sph_density_h(ctx, parts)
        sph.sph_forces(ctx, parts)
        return to_input_order(parts.numpy())
    finally:
        sph.sph_destroy(ctx)


@pytest.mark.parametrize("n", [14, 17])
def test_interface_correction_forces_match_oracle(sph, n):
    prob = slab_problem(n)
    p = oracle_params(prob)
    d = oracle.density_h(p, prob.pos, prob.m, prob.h0)
    ic = oracle.interface_correction(p, prob.pos, prob.m, d["h"], d["rho"], prob.u,
                                     prob.extra["mat"], prob.extra["r_gas"])
    f = oracle.forces(p, prob.pos, prob.vel, prob.m, d["h"], ic["rho_corr"], d["omega"], prob.u)
    f_off = oracle.forces(p, prob.pos, prob.vel, prob.m, d["h"], d["rho"], d["omega"], prob.u)
    g = _gpu(sph, prob, True)
    g_off = _gpu(sph, prob, False)
    assert rel_max(g["h"], d["h"]) < 1e-5 and rel_max(g["rho"], d["rho"]) < 1e-5
    errs = {k: norm_err(g[k], f[k]) for k in ("a", "dudt_h", "dudt_av", "divv")}
    print("interface correction n=%d" % n, {k: "%.2g" % v for k, v in errs.items()})
    for k, v in errs.items():
        assert v < 2e-4, (k, errs)
    assert rel_max(g["dt_i"], f["dt"]) < 1e-4
    # the correction is active: the forces differ from the uncorrected ones
    # (which match the oracle's uncorrected forces)
    assert norm_err(g_off["a"], f_off["a"]) < 2e-4
    assert norm_err(g["a"], g_off["a"]) > 1e-2


def test_interface_correction_needs_material_ids(sph):
    prob = slab_problem(8)
    prm = sph.Params.for_problem(prob, interface_correction=True, r_gas=prob.extra["r_gas"])
    parts = sph.Particles.from_problem(prob, "cuda:0")
    s = parts.c()
    s.mat = None
    import ctypes
    ctx = sph.sph_create(prm, prob.n)
    try:
        rc = sph.lib().sph_build_cells(ctx, ctypes.byref(s), None)
        assert rc == 1
    finally:
        sph.sph_destroy(ctx)
    with pytest.raises(sph.SphError):
        sph.sph_create(sph.Params(interface_correction=True, density="evolved"), 10)
    with pytest.raises(sph.SphError):
        sph.sph_create(sph.Params(interface_correction=True, precision="fp64"), 10)
