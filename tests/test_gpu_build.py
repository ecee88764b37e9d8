"""Particle order after sph_build_cells (Sec. 2.1: particles sorted along a
space-filling curve so that every cell is a contiguous range).

On a 16^3 lattice of cell centres in the unit box every particle sits in its
own block of 64^3 key cells, so the sorted order is the order of the curve
at level 4: for the Hilbert curve consecutive particles are face neighbours
(one lattice step along one axis), for the Morton curve their interleaved
lattice indices increase strictly."""
import numpy as np
import pytest

from paper_2511_11425_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2511_11425_gb300 as m
    m.lib()
    return m


def _lattice_order(sph, curve, periodic):
    n = 16
    prob = inputs.uniform(n=n, seed=5, jitter=0.0, vamp=0.0, periodic=periodic)
    params = sph.Params.for_problem(prob, curve=curve)
    ctx = sph.sph_create(params, prob.n)
    parts = sph.Particles.from_problem(prob)
    try:
        sph.sph_build_cells(ctx, parts)
        x = parts.pos().cpu().numpy()
        ids = parts.t["id"].cpu().numpy()
    finally:
        sph.sph_destroy(ctx)
    ijk = np.rint(x * n - 0.5).astype(np.int64)
    assert np.allclose(ijk, x * n - 0.5, atol=1e-9)
    assert sorted(ids.tolist()) == list(range(prob.n))
    assert np.array_equal(x, prob.pos[ids])
    return ijk


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0)])
def test_hilbert_order_steps_to_a_face_neighbour(sph, periodic):
    ijk = _lattice_order(sph, "hilbert", periodic)
    step = np.abs(np.diff(ijk, axis=0))
    assert np.all(step.sum(axis=1) == 1)
    assert len({tuple(r) for r in ijk.tolist()}) == len(ijk)


def test_morton_order_is_sorted_by_interleaved_index(sph):
    ijk = _lattice_order(sph, "morton", (1, 1, 1))

    def spread(v):
        out = np.zeros_like(v)
        for b in range(4):
            out |= ((v >> b) & 1) << (3 * b)
        return out
    key = spread(ijk[:, 0]) | (spread(ijk[:, 1]) << 1) | (spread(ijk[:, 2]) << 2)
    assert np.all(np.diff(key) > 0)


def test_tube_is_cut_into_cubes_visited_in_order(sph):
    """An elongated periodic box (4 x 1/4 x 1/4) is cut into 16 cubes of side
    1/4 along the tube; a 64 x 4 x 4 lattice (spacing 1/16) is ordered cube
    after cube, and inside a cube each step goes to a face neighbour."""
    import dataclasses
    import torch
    base = inputs.uniform(n=4, seed=5, jitter=0.0, vamp=0.0)
    ix, iy, iz = np.meshgrid(np.arange(64), np.arange(4), np.arange(4), indexing="ij")
    pos = (np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1) + 0.5) / 16.0
    n = len(pos)
    prob = dataclasses.replace(base, pos=pos, vel=np.zeros((n, 3)), u=np.ones(n),
                               m=np.full(n, 1.0 / n), h0=np.full(n, 2.5 / 16.0),
                               box_lo=(0.0, 0.0, 0.0), box_hi=(4.0, 0.25, 0.25))
    ctx = sph.sph_create(sph.Params.for_problem(prob), n)
    parts = sph.Particles.from_problem(prob)
    try:
        sph.sph_build_cells(ctx, parts)
        x = parts.pos().cpu().numpy()
    finally:
        sph.sph_destroy(ctx)
    ijk = np.rint(x * 16 - 0.5).astype(np.int64)
    cube = ijk[:, 0] // 4
    assert np.all(np.diff(cube) >= 0)
    step = np.abs(np.diff(ijk, axis=0)).sum(axis=1)
    same = cube[1:] == cube[:-1]
    assert np.all(step[same] == 1)
    assert np.all(step[~same] <= 4)


def _layout_checks(sph, prob, kappa_b=3.0, kappa_g=6.0, G=8):
    ctx = sph.sph_create(sph.Params.for_problem(prob), prob.n)
    parts = sph.Particles.from_problem(prob)
    try:
        sph.sph_build_cells(ctx, parts)
        first = sph.sph_bucket_layout(ctx)
        x = parts.pos().cpu().numpy()
        h = parts.t["h"].cpu().numpy()
    finally:
        sph.sph_destroy(ctx)
    cnt = np.diff(first)
    # slots cover every particle once, in order, at most 32 per bucket
    assert first[0] == 0 and first[-1] == prob.n
    assert np.all(cnt >= 0) and np.all(cnt <= 32)
    assert cnt.sum() == prob.n
    ext, gext = [], []
    for b in np.nonzero(cnt)[0]:
        xb = x[first[b]:first[b + 1]]
        ext.append(np.max(xb.max(0) - xb.min(0)) / h[first[b]:first[b + 1]].max())
    for g in range(0, len(cnt), G):
        lo, hi = first[g], first[min(g + G, len(cnt))]
        if hi > lo:
            xg = x[lo:hi]
            gext.append(np.max(xg.max(0) - xg.min(0)) / h[lo:hi].max())
    return cnt, np.array(ext), np.array(gext)


def test_bucket_layout_keeps_buckets_inside_small_cells(sph):
    """Free-surface sphere (random 1/r profile, open box): every bucket lies
    inside one cell of side <= 3 h and every group inside one of side
    <= 6 h (a box of that side fits within the cell); on an aligned periodic
    lattice the layout is the plain 32-particle chunking."""
    prob = inputs.collision(n_total=60000)
    cnt, ext, gext = _layout_checks(sph, prob)
    assert ext.max() <= 3.0 * 1.0001
    assert gext.max() <= 6.0 * 1.0001
    assert (cnt > 0).sum() <= 1.5 * prob.n / 32
    lat = inputs.sedov(n=32)
    cnt, ext, _ = _layout_checks(sph, lat)
    assert np.all(cnt[:lat.n // 32] == 32) and np.all(cnt[lat.n // 32:] == 0)
