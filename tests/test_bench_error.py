"""The bench's error report (bench.error_vs_oracle) on the CPU: fed the
oracle's own full solution it reports zero for every field, and an error
planted in one field shows up in that field only, at its size."""
import numpy as np

import bench
import oracle
from oracle import build as obuild
from paper_2511_11425_gb300 import inputs


def _full_solution(prob, p):
    d = oracle.density_h(p, prob.pos, prob.m, prob.h0)
    f = oracle.forces(p, prob.pos, prob.vel, prob.m, d["h"], d["rho"], d["omega"], prob.u)
    return {"h": d["h"], "rho": d["rho"], "omega": d["omega"], "a": f["a"],
            "dudt_h": f["dudt_h"], "dudt_av": f["dudt_av"], "divv": f["divv"]}


def test_error_report_is_exact_and_field_by_field():
    obuild.build()
    prob = inputs.uniform(n=12, seed=9, jitter=0.3, vamp=0.3)
    p = oracle.Params(gamma=prob.gamma, alpha=prob.alpha, beta=prob.beta, box_lo=prob.box_lo,
                      box_hi=prob.box_hi, periodic=prob.periodic)
    full = _full_solution(prob, p)
    e = bench.error_vs_oracle(prob, full, p)
    fields = ("h", "rho", "omega", "a", "dudt_h", "dudt_av", "divv")
    assert all(e[k] < 1e-12 for k in fields), e
    assert e["sinks"] > 100 and e["neighbourhood"] >= e["sinks"]
    planted = dict(full)
    planted["rho"] = full["rho"] * (1.0 + 1e-4)
    e2 = bench.error_vs_oracle(prob, planted, p)
    assert abs(e2["rho"] - 1e-4) < 1e-9
    assert all(e2[k] < 1e-12 for k in fields if k != "rho")


def test_error_report_normalises_by_the_whole_field():
    # the sample holds the particles where the field is largest, so the max
    # norm is the whole field's, not the clusters'
    obuild.build()
    prob = inputs.uniform(n=12, seed=9, jitter=0.3, vamp=0.3)
    p = oracle.Params(gamma=prob.gamma, alpha=prob.alpha, beta=prob.beta, box_lo=prob.box_lo,
                      box_hi=prob.box_hi, periodic=prob.periodic)
    full = _full_solution(prob, p)
    k = int(np.argmax(np.abs(full["divv"])))
    planted = dict(full)
    planted["divv"] = full["divv"].copy()
    planted["divv"][k] += 1e-3 * full["divv"][k]
    e = bench.error_vs_oracle(prob, planted, p)
    assert abs(e["divv"] - 1e-3) < 1e-9
    assert set(bench._field_maxima(full).tolist()) <= set(range(prob.n))
    assert len(bench._field_maxima(full)) == 4 * bench.FIELD_MAXIMA_PER_FIELD
