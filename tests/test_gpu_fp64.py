"""The FP64 form (sph_params.precision = SPH_PRECISION_FP64) against the FP64
oracle, through the C ABI.

The FP64 form takes the pair sums, the h iteration and the force
accumulators in FP64; h, rho, Omega and the outputs are still stored in the
FP32 arrays of sph_particles, so its error against the oracle is set by
that storage: about 1e-7 relative, far inside the tolerances (1e-5 for h,
rho, Omega; 2e-4 of the field's max norm for a, du/dt, div v).  The mixed
form of the same inputs is evaluated beside it, and the FP64 form must be
closer to the oracle on the cancelling PdV sum of the Kelvin-Helmholtz
layer."""
import numpy as np
import pytest

from helpers import gpu_evaluate, norm_err, oracle_params, oracle_sampled, rel_max
from paper_2511_11425_gb300 import inputs
from test_gpu_parity import _assert_errs, _full_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2511_11425_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("n,periodic,kernel,nngb", [(15, (1, 1, 1), "wc2", 64),
                                                    (13, (0, 0, 0), "wc2", 64),
                                                    (14, (1, 1, 1), "wc6", 200),
                                                    (14, (1, 1, 1), "m4", 32)])
def test_fp64_form_parity(sph, n, periodic, kernel, nngb):
    prob = inputs.uniform(n=n, seed=300 + n, jitter=0.35, vamp=0.4, periodic=periodic)
    prob.kernel, prob.n_ngb = kernel, nngb
    prob.h0 = prob.h0 * (nngb / 64.0) ** (1 / 3)
    # a Newton tolerance far below FP32 resolution: the error left is the
    # FP32 storage of h, rho, Omega between the passes
    g = gpu_evaluate(prob, sph.Params.for_problem(prob, precision="fp64", h_rel_tol=1e-10))
    errs, d, f = _full_parity(prob, g)
    print("fp64 form", kernel, periodic, {k: "%.2g" % v for k, v in errs.items()})
    _assert_errs(errs)
    assert errs["h"] < 3e-7 and errs["rho"] < 1e-6 and errs["omega"] < 1e-6, errs
    for k in ("a", "dudt_h", "dudt_av", "divv"):
        assert errs[k] < 2e-6, (k, errs)
    assert int(np.sum(g["nngb"] != d["nngb"])) <= 2


def test_fp64_form_sod_and_steps(sph):
    # the Sod tube at t = 0, then 5 steps of both forms from the same state
    prob = inputs.sod()
    g = gpu_evaluate(prob, sph.Params.for_problem(prob, precision="fp64"))
    errs, d, f = _full_parity(prob, g)
    _assert_errs(errs)
    sims = {m: sph.Simulation(prob, sph.Params.for_problem(prob, precision=m))
            for m in ("mixed", "fp64")}
    try:
        for _ in range(5):
            dts = {m: s.step(2e-4) for m, s in sims.items()}
        out = {m: s.parts.numpy() for m, s in sims.items()}
    finally:
        for s in sims.values():
            s.close()
    a = {m: np.argsort(o["id"]) for m, o in out.items()}
    for k in ("x0", "u"):
        x_m = out["mixed"][k][a["mixed"]]
        x_d = out["fp64"][k][a["fp64"]]
        assert np.max(np.abs(x_m - x_d)) <= 1e-6 * np.max(np.abs(x_d)), k


def test_fp64_form_kelvin_helmholtz_pdv_sum(sph):
    # 32^3 shear layer: the PdV sum cancels across the shear; the FP64 form
    # meets the oracle far inside the mixed form's error
    prob = inputs.kh(n=32)
    rng = np.random.default_rng(4)
    centres = [[0.3, 0.25, 0.6], [0.7, 0.75, 0.2]] + list(rng.random((1, 3)))
    L = 1.0
    sinks = []
    for c in centres:
        dd = prob.pos - np.asarray(c)
        dd -= L * np.round(dd / L)
        sinks.extend(np.argsort((dd * dd).sum(1))[:12])
    sinks = np.unique(np.array(sinks))
    o = oracle_sampled(prob, oracle_params(prob), sinks)
    errs = {}
    for mode in ("mixed", "fp64"):
        g = gpu_evaluate(prob, sph.Params.for_problem(prob, precision=mode))
        errs[mode] = {k: norm_err(g[k][sinks], o[k]) for k in ("a", "dudt_h", "divv")}
        errs[mode]["h"] = rel_max(g["h"][sinks], o["h"])
    print("KH 32^3 errors", errs)
    for mode in errs:
        assert errs[mode]["h"] < 1e-5 and errs[mode]["dudt_h"] < 2e-4, (mode, errs)
    assert errs["fp64"]["dudt_h"] < 1e-5 and errs["fp64"]["divv"] < 1e-5, errs
