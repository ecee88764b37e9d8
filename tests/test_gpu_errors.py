"""Error paths of a step, made on the host: the status a failing step
returns and the state it leaves.

A step that fails (sph_step returns an error) must leave the particles'
positions, velocities and internal energies as they were: the kernels that
change the state check the device status word and skip their work once an
earlier kernel of the same step raised an error.  The build still reorders
the arrays into curve order, so the state is compared in the caller's
particle order (by id)."""
import numpy as np
import pytest

from helpers import to_input_order
from paper_2511_11425_gb300 import inputs
from test_gpu_overflow import heavy_lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2511_11425_gb300 as m
    m.lib()
    return m


def _state(parts):
    g = to_input_order(parts.numpy())
    return g["x"].copy(), g["v"].copy(), g["u"].copy()


def _assert_unchanged(before, parts):
    after = _state(parts)
    for a, b, name in zip(before, after, ("x", "v", "u")):
        assert np.array_equal(a, b), name


def test_newton_cap_reports_noconv_and_keeps_the_state(sph):
    # one Newton iteration from a seed at a fifth of the converged h cannot
    # reach the tolerance: SPH_ERR_NOCONV
    prob = inputs.uniform(n=10, seed=3, jitter=0.3, vamp=0.3)
    prob.h0 = 0.2 * prob.h0
    prm = sph.Params.for_problem(prob, max_newton=1)
    parts = sph.Particles.from_problem(prob, "cuda:0")
    before = _state(parts)
    ctx = sph.sph_create(prm, prob.n)
    try:
        with pytest.raises(sph.SphError) as e:
            sph.sph_step(ctx, parts, 1e-3)
        assert e.value.code == 4, e.value
    finally:
        sph.sph_destroy(ctx)
    _assert_unchanged(before, parts)


def test_full_list_arena_reports_capacity_and_keeps_the_state(sph):
    # the heavy particle's walk group needs about 1,200 overflow entries; an
    # arena of 64 cannot hold them: SPH_ERR_CAPACITY
    prob, _ = heavy_lattice()
    parts = sph.Particles.from_problem(prob, "cuda:0")
    before = _state(parts)
    ctx = sph.sph_create(sph.Params.for_problem(prob), prob.n)
    try:
        sph.sph_set_list_arena(ctx, 64)
        with pytest.raises(sph.SphError) as e:
            sph.sph_step(ctx, parts, 1e-4)
        assert e.value.code == 3, e.value
        _assert_unchanged(before, parts)
        # a large enough arena lets the same context step
        sph.sph_set_list_arena(ctx, 1 << 20)
        sph.sph_step(ctx, parts, 1e-4)
        x, _, _ = _state(parts)
        assert not np.array_equal(x, before[0])
    finally:
        sph.sph_destroy(ctx)
    with pytest.raises(sph.SphError) as e:
        ctx = sph.sph_create(sph.Params(), 10)
        try:
            sph.sph_set_list_arena(ctx, -1)
        finally:
            sph.sph_destroy(ctx)
    assert e.value.code == 1


def test_nonfinite_velocity_reports_and_keeps_the_state(sph):
    prob = inputs.uniform(n=8, seed=5, jitter=0.3, vamp=0.3)
    parts = sph.Particles.from_problem(prob, "cuda:0")
    parts.t["u"][3] = -1.0      # negative internal energy: non-finite sound speed
    before = _state(parts)
    ctx = sph.sph_create(sph.Params.for_problem(prob), prob.n)
    try:
        with pytest.raises(sph.SphError) as e:
            sph.sph_step(ctx, parts, 1e-3)
        assert e.value.code == 5, e.value
    finally:
        sph.sph_destroy(ctx)
    _assert_unchanged(before, parts)
