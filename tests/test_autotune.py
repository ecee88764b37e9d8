"""Host logic of the autotuner: the coordinate descent, the cache keyed by
GPU and configuration class, and that tuned settings only touch the layout
knobs.  The GPU test runs the real timer and checks that a tuned step gives
the same fields as a default one."""
import numpy as np
import pytest

from paper_2511_11425_gb300 import Params, autotune, inputs


def test_coordinate_descent_finds_the_separable_optimum():
    best = {"curve": "morton", "bucket_cell": 4.0, "group_log": 2, "list_margin": 0.05}
    cost = {"curve": {"hilbert": 1.0, "morton": 0.0},
            "bucket_cell": {3.0: 2.0, 2.0: 3.0, 4.0: 0.0},
            "group_log": {3: 1.0, 2: 0.0},
            "list_margin": {0.1: 1.0, 0.05: 0.0, 0.2: 2.0}}
    calls = []

    def measure(k):
        calls.append(dict(k))
        return 10.0 + sum(cost[n][k[n]] for n in cost)
    start = {"curve": "hilbert", "bucket_cell": 3.0, "group_log": 3, "list_margin": 0.1,
             "resort_period": 1}
    cost["resort_period"] = {1: 1.0, 4: 0.0, 8: 0.5, 16: 0.7}
    best["resort_period"] = 4
    knobs, t, tried = autotune.coordinate_descent(measure, start)
    assert knobs == best and t == 10.0
    assert len(tried) == len(calls) == 1 + 3 + 1 + 2 + 1 + 2


def test_small_gains_are_not_taken():
    def measure(k):
        return 100.0 - (1.0 if k["curve"] == "morton" else 0.0)   # 1 % faster only
    start = {"curve": "hilbert", "bucket_cell": 3.0, "group_log": 3, "list_margin": 0.1,
             "resort_period": 1}
    knobs, _, _ = autotune.coordinate_descent(measure, start)
    assert knobs["curve"] == "hilbert"


def test_cache_is_keyed_by_gpu_and_configuration(tmp_path):
    calls = []

    def measure(parts, plist, offsets):
        calls.append(plist[0])
        return 5.0 if plist[0].group_log == 2 else 6.0

    class P:
        n = 4096
    path = str(tmp_path / "tune.json")
    prm = Params(periodic=(1, 1, 1))
    t = autotune.Autotuner(path, measure=measure)
    got = t.tune(P(), prm, device_name="GPU-A")
    assert got.group_log == 2 and not t.report["cached"]
    n1 = len(calls)
    got2 = t.tune(P(), prm, device_name="GPU-A")          # cached: no timing
    assert len(calls) == n1 and got2 == got and t.report["cached"]
    t.tune(P(), prm, device_name="GPU-B")                 # another GPU: timed again
    assert len(calls) == 2 * n1
    t.tune(P(), Params(periodic=(0, 0, 0)), device_name="GPU-A")   # open box: timed again
    assert len(calls) == 3 * n1
    t.tune(P(), prm, device_name="GPU-A", force=True)
    assert len(calls) == 4 * n1
    # a batch keys on its instance count and returns one Params per instance
    plist = t.tune(P(), [prm] * 4, offsets=[0, 1, 2, 3, 4], device_name="GPU-A")
    assert len(plist) == 4 and all(p.group_log == 2 for p in plist)
    assert autotune.config_class(4096, [prm], "G") != autotune.config_class(4096, [prm] * 4, "G")
    assert autotune.config_class(4096, [prm], "G") != autotune.config_class(65536, [prm], "G")


def test_tuned_params_change_only_layout_knobs():
    p = Params.for_problem(inputs.sod())
    q = autotune.with_knobs(p, {"curve": "morton", "bucket_cell": 4.0, "group_log": 2,
                                "list_margin": 0.2, "resort_period": 4})
    assert q.group_cell == 8.0 and q.curve == "morton" and q.resort_period == 4
    for f in ("gamma", "alpha", "beta", "n_ngb", "kernel", "box_lo", "box_hi", "periodic",
              "eta_courant", "h_rel_tol"):
        assert getattr(q, f) == getattr(p, f)


@pytest.mark.gpu
def test_tuned_step_matches_default_step(tmp_path):
    import torch
    import paper_2511_11425_gb300 as sph
    from helpers import norm_err, to_input_order
    assert torch.cuda.is_available()
    prob = inputs.uniform(n=20, seed=17, vamp=0.3, jitter=0.3)
    base = sph.Params.for_problem(prob)
    parts = sph.Particles.from_problem(prob)
    tuner = autotune.Autotuner(str(tmp_path / "t.json"), steps=1, warmup=1)
    tuned = tuner.tune(parts, base, force=True)
    assert len(tuner.report["tried"]) >= 8
    assert all(r["ms_per_step"] > 0 for r in tuner.report["tried"])
    out = {}
    for name, prm in (("default", base), ("tuned", tuned)):
        s = sph.Simulation(prob, prm)
        try:
            s.step()
            out[name] = to_input_order(s.parts.numpy())
        finally:
            s.close()
    assert np.max(np.abs(out["tuned"]["h"] / out["default"]["h"] - 1)) < 1e-5
    assert norm_err(out["tuned"]["a"], out["default"]["a"]) < 1e-5
