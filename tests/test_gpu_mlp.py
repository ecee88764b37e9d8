"""The learned seed of the h iteration on the GPU against the FP64 oracle
(oracle.mlp): loss gradients of the FP32 training kernels, Adam steps,
the bfloat16 tensor-core inference (exactly, on a network built by hand,
and within the rounding bound on random weights), and the recording of
training samples from the simulation's own converged h."""
import numpy as np
import pytest

from helpers import to_input_order
from oracle import mlp
from paper_2511_11425_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2511_11425_gb300 as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def ctx(sph):
    prob = inputs.uniform(n=8, seed=1)
    c = sph.sph_create(sph.Params.for_problem(prob), prob.n)
    yield c
    sph.sph_destroy(c)


def _weights(seed, w3_scale=0.3):
    w = inputs.mlp_init(seed)
    rng = np.random.default_rng(seed)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(w)
    W3 = rng.normal(0.0, w3_scale, 32)
    b1 = rng.normal(0.0, 0.1, 32)
    b2 = rng.normal(0.0, 0.1, 32)
    return mlp.pack(W1, b1, W2, b2, W3, 0.05).astype(np.float32).astype(np.float64)


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0.0, 1.0, (n, 4)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]).astype(np.float32)
    return X, y


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [1, 1000, 300001])
def test_gradient_matches_oracle(sph, ctx, n):
    w = _weights(3)
    X, y = _samples(n, n)
    sph.sph_mlp_set_weights(ctx, w)
    g, loss = sph.sph_mlp_grad(ctx, _dev(X), _dev(y))
    lo, go = mlp.loss_and_grad(w, X.astype(np.float64), y.astype(np.float64))
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.max(np.abs(g - go)) <= 1e-4 * np.max(np.abs(go))
    # gradient blocks of every layer are non-trivial
    assert np.max(np.abs(go[:128])) > 0 and np.max(np.abs(go[160:1184])) > 0


def test_adam_steps_match_oracle(sph, ctx):
    w0 = _weights(4)
    X, y = _samples(777, 5)
    sph.sph_mlp_set_weights(ctx, w0)
    sph.sph_mlp_load_samples(ctx, _dev(X), _dev(y))
    assert sph.sph_mlp_samples(ctx) == 777
    lr = 1e-3
    l0, l3 = sph.sph_mlp_train(ctx, 4, batch=0, lr=lr)
    got = sph.sph_mlp_get_weights(ctx).astype(np.float64)
    w = w0.copy()
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    losses = []
    for t in range(1, 5):
        loss, g = mlp.loss_and_grad(w, X.astype(np.float64), y.astype(np.float64))
        losses.append(loss)
        w, m, v = mlp.adam_step(w, g, m, v, t, lr)
    assert abs(l0 - losses[0]) <= 1e-5 * losses[0] and abs(l3 - losses[3]) <= 1e-5 * losses[3]
    moved = np.abs(w - w0) > 0.5 * lr          # parameters Adam moves by ~lr per step
    assert moved.sum() > 900
    assert np.max(np.abs(got - w)[moved]) <= 0.02 * lr
    # parameters with near-zero gradients follow FP32 rounding noise, within
    # the step bound of Adam
    assert np.max(np.abs(got - w)) <= 2 * lr


def _hand_network(seed):
    """y = x0 - 2 x1 + 0.5 x2 + 4 x3 + 0.25 through ReLU pairs placed on
    random hidden units of both layers."""
    rng = np.random.default_rng(seed)
    p1 = rng.permutation(32)[:8]
    p2 = rng.permutation(32)[:8]
    W1 = np.zeros((32, 4)); W2 = np.zeros((32, 32)); W3 = np.zeros(32)
    coef = [1.0, -2.0, 0.5, 4.0]
    for a in range(4):
        W1[p1[2 * a], a] = 1.0
        W1[p1[2 * a + 1], a] = -1.0
        W2[p2[2 * a], p1[2 * a]] = 1.0
        W2[p2[2 * a + 1], p1[2 * a + 1]] = 1.0
        W3[p2[2 * a]] = coef[a]
        W3[p2[2 * a + 1]] = -coef[a]
    return mlp.pack(W1, np.zeros(32), W2, np.zeros(32), W3, 0.25), np.array(coef)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tensor_core_inference_is_exact_on_a_hand_built_network(sph, ctx, seed):
    w, coef = _hand_network(seed)
    sph.sph_mlp_set_weights(ctx, w)
    rng = np.random.default_rng(seed + 10)
    X = (np.round(rng.uniform(-8, 8, (1037, 4)) * 4) / 4).astype(np.float32)
    y = sph.sph_mlp_infer(ctx, _dev(X)).cpu().numpy()
    assert np.array_equal(y.astype(np.float64), X.astype(np.float64) @ coef + 0.25)


def test_tensor_core_inference_matches_bf16_oracle(sph, ctx):
    w = _weights(6, 0.5)
    sph.sph_mlp_set_weights(ctx, w)
    X, _ = _samples(4133, 7)
    y = sph.sph_mlp_infer(ctx, _dev(X)).cpu().numpy().astype(np.float64)
    ref = mlp.infer_bf16(w, X.astype(np.float64))
    W1, b1, W2, b2, W3, b3 = mlp.unpack(w)
    a2 = np.maximum(np.maximum(X @ W1.T + b1, 0) @ W2.T + b2, 0)
    scale = a2 @ np.abs(W3) + 1e-3
    # FP32 sums in another order can move a hidden activation by one
    # bfloat16 step (2^-8 relative) before the output layer
    assert np.all(np.abs(y - ref) <= 2.0 ** -6 * scale)
    assert np.mean(np.abs(y - ref)) <= 1e-3 * np.mean(np.abs(ref))
    # and the rounding itself is small against the FP64 network
    assert np.mean(np.abs(y - mlp.forward(w, X.astype(np.float64)))) <= 0.02 * np.mean(np.abs(ref))


def test_recorded_samples_pair_inputs_with_the_converged_h(sph):
    """One recorded step of a shearing jittered lattice, run phase by phase:
    the samples are exactly the oracle's (features, target) of the particles,
    built from the seed, converged h, div v, neighbour count and step sizes
    read back between the phases."""
    prob = inputs.uniform(n=12, seed=21, vamp=0.5, jitter=0.3)
    sim = sph.Simulation(prob)
    try:
        dt_old = sim.step()
        sph.sph_mlp_record(sim.ctx, True, capacity=100000, stride=1)
        sph.sph_build_cells(sim.ctx, sim.parts)
        seed_b = sim.parts.t["h"].cpu().numpy().astype(np.float64)
        sph.sph_density_h(sim.ctx, sim.parts)
        h_b = sim.parts.t["h"].cpu().numpy().astype(np.float64)
        nngb = sim.parts.t["nngb"].cpu().numpy().astype(np.float64)
        sph.sph_forces(sim.ctx, sim.parts)
        divv = sim.parts.t["divv"].cpu().numpy().astype(np.float64)
        ids_b = sim.parts.t["id"].cpu().numpy()
        dt = sph.sph_kdk_step(sim.ctx, sim.parts)
        assert sph.sph_mlp_samples(sim.ctx) == 0
        sph.sph_build_cells(sim.ctx, sim.parts)
        sph.sph_density_h(sim.ctx, sim.parts)
        h_c = np.empty(prob.n)
        h_c[sim.parts.t["id"].cpu().numpy()] = sim.parts.t["h"].cpu().numpy()
        gx, gy = sph.sph_mlp_get_samples(sim.ctx)
    finally:
        sim.close()
    X = mlp.features(dt, divv, nngb, prob.n_ngb, h_b, seed_b, dt_old)
    Y = mlp.target(h_c[ids_b], h_b, X)
    assert len(gy) == prob.n                         # stride 1: every particle
    assert np.std(X[:, 0]) > 0 and np.std(X[:, 1]) > 0 and np.std(X[:, 2]) > 0
    assert np.all(X[:, 3] == X[0, 3]) and X[0, 3] != 0
    # match every sample to its particle (nearest in (x, y) space)
    ref = np.concatenate([X, Y[:, None]], axis=1)
    got = np.concatenate([gx, gy[:, None]], axis=1).astype(np.float64)
    sc = np.maximum(np.std(ref, axis=0), 1e-3)
    used = np.zeros(len(ref), dtype=bool)
    for row in got:
        d = np.max(np.abs((ref - row) / sc), axis=1)
        j = int(np.argmin(np.where(used, np.inf, d)))
        used[j] = True
        assert np.all(np.abs(ref[j] - row) <= 1e-4 * np.abs(ref[j]) + 2e-5), (row, ref[j])
    assert used.all()


def _phases(sph, sim):
    """One step phase by phase; returns what the seed of the next step is
    made from (in the order of this step) and the dt pair."""
    sph.sph_build_cells(sim.ctx, sim.parts)
    seed = sim.parts.t["h"].cpu().numpy().astype(np.float64)
    sph.sph_density_h(sim.ctx, sim.parts)
    h = sim.parts.t["h"].cpu().numpy().astype(np.float64)
    iters = sim.parts.t["iters"].cpu().numpy().astype(np.float64)
    nngb = sim.parts.t["nngb"].cpu().numpy().astype(np.float64)
    sph.sph_forces(sim.ctx, sim.parts)
    divv = sim.parts.t["divv"].cpu().numpy().astype(np.float64)
    return seed, h, iters, nngb, divv


def test_kick_writes_the_learned_seed(sph):
    """In SPH_SEED_MLP mode the kick leaves h at the oracle's seed built from
    the bfloat16 network output on the oracle's features."""
    prob = inputs.uniform(n=12, seed=23, vamp=0.5, jitter=0.3)
    sim = sph.Simulation(prob)
    w = _weights(8, 0.5)
    try:
        dt_old = sim.step()
        sph.sph_mlp_set_weights(sim.ctx, w)
        sph.sph_mlp_set_seed_mode(sim.ctx, "mlp")
        seed, h, _, nngb, divv = _phases(sph, sim)
        dt = sph.sph_kdk_step(sim.ctx, sim.parts)
        got = sim.parts.t["h"].cpu().numpy().astype(np.float64)
    finally:
        sim.close()
    X = mlp.features(dt, divv, nngb, prob.n_ngb, h, seed, dt_old)
    X32 = X.astype(np.float32).astype(np.float64)
    y = mlp.infer_bf16(w, X32)
    ref = mlp.seed(h, X32, y, tol=1e-6)
    assert np.mean(np.abs(ref / h - 1.0)) > 1e-3       # the network moved the seeds
    W1, b1, W2, b2, W3, b3 = mlp.unpack(w)
    a2 = np.maximum(np.maximum(X32 @ W1.T + b1, 0) @ W2.T + b2, 0)
    tol = 2.0 ** -6 * (a2 @ np.abs(W3) + 1e-3) / mlp.Y_SCALE + 1e-6
    assert np.all(np.abs(np.log(got / ref)) <= tol)


def test_trained_seed_is_closer_to_the_converged_h(sph):
    """Train on 20 recorded steps of a Kelvin-Helmholtz shear layer, then run
    the same 6 steps from the same state with the continuity seed (a copy of
    the state) and with the learned seed (the training context, dead zone
    included): the learned seeds are closer to the h the iteration converges
    to, the iteration needs no more passes, and the converged fields agree
    to within a few times the iteration's tolerance.  The iteration ends with
    its estimate of the remaining error below h_rel_tol (the quadratic step
    rule of the density pass), so each converged h lies up to about tol from
    its root; the two runs start each evaluation from different seeds and
    drift apart over the 6 steps."""
    tol = 1e-5
    prob = inputs.kh(n=32)
    params = sph.Params.for_problem(prob, h_rel_tol=tol)
    sim = sph.Simulation(prob, params)
    ref = sph.Simulation(prob, params)
    try:
        sim.step()
        sph.sph_mlp_record(sim.ctx, True, capacity=1 << 20, stride=1)
        for _ in range(20):
            dt = sim.step()
        sph.sph_mlp_record(sim.ctx, False)
        assert sph.sph_mlp_samples(sim.ctx) > 15 * prob.n
        sph.sph_mlp_set_weights(sim.ctx, inputs.mlp_init(3))
        l0, _ = sph.sph_mlp_train(sim.ctx, 2000, batch=8192, lr=2e-3, seed=1)
        _, l1 = sph.sph_mlp_train(sim.ctx, 2000, batch=8192, lr=5e-4, seed=2)
        assert l1 < 0.05 * l0
        for k, v in sim.parts.t.items():
            ref.parts.t[k].copy_(v)
        sph.sph_set_dt_old(ref.ctx, dt)
        sph.sph_mlp_set_seed_mode(sim.ctx, "mlp")
        runs = {}
        for mode, s in (("analytic", ref), ("mlp", sim)):
            err, its = [], []
            for _ in range(6):
                seed, h, iters, _, _ = _phases(sph, s)
                sph.sph_kdk_step(s.ctx, s.parts)
                err.append(np.abs(np.log(h / seed)))
                its.append(iters)
            runs[mode] = (np.concatenate(err[1:]), np.concatenate(its[1:]),
                          to_input_order(s.parts.numpy()))
    finally:
        sim.close()
        ref.close()
    ea, ia, ga = runs["analytic"]
    em, im, gm = runs["mlp"]
    assert np.mean(em) < 0.8 * np.mean(ea)
    assert np.mean(im) <= np.mean(ia) + 0.01
    assert np.max(np.abs(gm["h"] / ga["h"] - 1.0)) < 20 * tol
    assert np.max(np.abs(gm["rho"] / ga["rho"] - 1.0)) < 60 * tol
