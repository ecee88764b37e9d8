"""The allocation-free conserved totals (sph_reduce_conserved_noalloc) agree
with the context-based sph_reduce_conserved.

The entry point serves callers that cannot allocate device memory, so it keeps
its block partials in a fixed device array that persists between calls; this
file is collected last so that a failure here cannot hide the other tests.
Two calls in a row on different data check that the persistent array carries
nothing from one call into the next."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _reference(sph, prob, parts):
    ctx = sph.sph_create(sph.Params.for_problem(prob), prob.n)
    try:
        return np.array(sph.sph_reduce_conserved(ctx, parts))
    finally:
        sph.sph_destroy(ctx)


def test_noalloc_totals_match_context_totals_twice():
    import torch

    import oracle
    import paper_2511_11425_gb300 as sph
    from paper_2511_11425_gb300 import inputs

    assert torch.cuda.is_available()
    lib = sph.lib()
    out = torch.zeros(9, dtype=torch.float64, device="cuda:0")
    # first a multi-block problem, then a smaller one: the second call must not
    # see the first call's partials
    for prob in (inputs.sedov(n=48, seed=3), inputs.uniform(n=9, seed=4, vamp=0.3)):
        parts = sph.Particles.from_problem(prob, "cuda:0")
        ref = _reference(sph, prob, parts)
        out.fill_(float("nan"))
        s = parts.c()
        rc = lib.sph_reduce_conserved_noalloc(ctypes.byref(s), ctypes.c_void_p(out.data_ptr()),
                                              None)
        assert rc == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-15), (got, ref)
        # and against the FP64 oracle's totals of the same state (masses as
        # the device holds them, in float32)
        g = parts.numpy()
        x = np.stack([g["x0"], g["x1"], g["x2"]], 1)
        v = np.stack([g["v0"], g["v1"], g["v2"]], 1)
        o = oracle.conserved(x, v, g["m"].astype(np.float64), g["u"])
        scale = np.array([o[0]] + [np.max(np.abs(o[1:4])) + 1e-300] * 3 +
                         [np.max(np.abs(o[4:7])) + 1e-300] * 3 + [o[7], o[8]])
        assert np.all(np.abs(got - o) <= 1e-12 * np.maximum(scale, np.abs(o))), (got, o)


def test_noalloc_rejects_too_many_particles():
    import paper_2511_11425_gb300 as sph
    s = sph.c_particles()
    s.n = 8_388_609
    assert sph.lib().sph_reduce_conserved_noalloc(ctypes.byref(s), ctypes.c_void_p(16), None) == 3
