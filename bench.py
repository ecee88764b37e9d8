"""Benchmark of the SPH hot path on GB300 (one JSON line on stdout).

Workload: the Sedov-Taylor blast of the paper's test suite (Sec. 3.3) on a
64^3 = 262,144-particle jittered periodic lattice, Wendland C2 with 64
neighbours, alpha = 1, beta = 2, gamma = 5/3, starting at t = 0.  One step =
sph_step: Morton sort + bounds tree, density/h Newton pass, force pass,
kick-drift-kick with the Courant step (every row of the hot path), plus the
conserved-totals reduction.  --workload kh128 times the Kelvin-Helmholtz
shear layer (Sec. 3.8 setting) on 128^3 = 2,097,152 particles instead.

  value       particle-steps/s with the state resident in HBM; each timed step
              is one replay of the captured step (CUDA graph, conserved totals
              included) bracketed by CUDA events on its stream, and a 256 MiB
              buffer is written between steps so no step starts with a warm L2
  e2e         the same metric through sph_step_host (replaying the step that
              sph_step_host_capture recorded): the step's input arrays copied
              from pinned host memory, stepped, and every array copied back,
              all inside the timed region
  roofline    the dominant pair kernel against the FP32 pipe peak
              (152 SMs x 128 lanes x 2 flop x 2.07 GHz), algorithmic flops only
  cpu_baseline the FP64 oracle on a bounded sample of the same state
  error_vs_oracle  per-field error of the GPU path against the oracle on
              sampled sinks of the stepped state (the 'stated error' of the
              metric), computed in the oracle's leg

--impl reference times the oracle (the deliberately slow FP64 brute force)
on the same workload and metric.  Under torchrun every rank runs its own
independent replica (weak scaling, no data exchange); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP32_LANES = 128      # FP32 lanes per SM (4 sub-partitions x 32)
SM_MAX_GHZ = 2.070    # maximum SM clock of the GB300 (nvidia-smi clocks.max.sm)


def fp32_peak_tflops(sms):
    """Derived FP32 peak: SMs x 128 lanes x 2 flop (FMA) x maximum SM clock."""
    return sms * FP32_LANES * 2 * SM_MAX_GHZ / 1000.0


def fma_probe(stream):
    """Measured FP32 FMA throughput (TFLOP/s) and SM count of the current
    device, from the benchmark's own probe library (_fma_probe.so, built
    beside libsph but not part of it); (None, None) if it cannot run."""
    import ctypes as C
    import paper_2511_11425_gb300 as sph
    path = os.path.join(os.path.dirname(sph.LIB_PATH), "_fma_probe.so")
    try:
        L = C.CDLL(path)
    except OSError:
        return None, None
    L.fma_probe_tflops.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p]
    L.fma_probe_tflops.restype = C.c_int
    t, n = C.c_double(), C.c_int()
    handle = stream.cuda_stream if stream is not None else None
    if L.fma_probe_tflops(C.byref(t), C.byref(n), C.c_void_p(handle)) != 0:
        return None, None
    return t.value, n.value
# Algorithmic flops per unit (FMA = 2; add, mul, divide, rsqrt = 1; compares,
# selects and min/max not counted), tallied from the pair loops:
#  density pair (Wendland C2): separation 3, r^2 5, r 2, q 1, w(q) 6,
#    w'(q)/q 3, S_w 2, S_q 4                                          = 26
#  force pair without viscosity: separation 3, r^2 5, r 2, 1/h_j^2 1,
#    q_i q_j 2, F_i 5, F_j 8, v_ij 3, v_ij.r_ij 5, coefficient 5,
#    sink a 1+6, sink S 3, source a+S 9 (incl. the four adds)          = 61 (incl. 1/h_j
#    staged once per source, counted per pair as the method needs it)
#  viscosity on top: h, c, rho averages 6, mu 5, Pi 6, du/dt|Pi 3,
#    sink du 2, source du 2                                            = 24
FLOPS_DENSITY_PAIR = 26      # one useful (r < h) pair evaluation of one Newton pass
FLOPS_FORCE_PAIR = 61        # one unordered pair, pressure and PdV terms, both sides
FLOPS_FORCE_AV = 24          # extra flops of a pair with active viscosity
METRIC = "SPH particle-steps/s"
UNIT = "particle-steps/s"


WORKLOADS = {
    "sedov64": "sedov_taylor_64^3 (262,144 particles, periodic unit box, t from 0)",
    "kh128": "kelvin_helmholtz_128^3 (2,097,152 particles, periodic unit box, t from 0)",
}
_WORKLOAD = ["sedov64"]  # set from --workload


def _workload(rank=0):
    from paper_2511_11425_gb300 import inputs
    if _WORKLOAD[0] == "kh128":
        return inputs.kh(n=128, seed=2511 + rank)
    return inputs.sedov(n=64, seed=2511 + rank)


def _config(prob, extra=None):
    c = {"workload": WORKLOADS[_WORKLOAD[0]],
         "particles": prob.n, "kernel": "wendland_c2", "n_ngb": 64, "gamma": prob.gamma,
         "alpha": prob.alpha, "beta": prob.beta,
         "precision": "fp32 pair arithmetic on cell-relative offsets, fp64 positions and "
                      "kick-drift-kick",
         "l2": "flushed between timed steps (256 MiB write)"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except (ValueError, IndexError):
                continue
            for k, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _ncu_record(kernel_file, kernel_name):
    """The committed ncu summary of a kernel (profiles/traffic.json), if it
    still describes the current source of that kernel and was taken on the
    workload being timed."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel_name)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("bench_workload") != _WORKLOAD[0]:
        return None
    src = open(os.path.join(ROOT, "paper_2511_11425_gb300", "csrc", kernel_file), "rb").read()
    if hashlib.sha256(src).hexdigest()[:16] != rec.get("source_sha"):
        return None
    return rec


def _traffic_for(kernel_file, kernel_name):
    """DRAM bytes per launch from the committed ncu summary, if it still
    describes the current source of that kernel."""
    rec = _ncu_record(kernel_file, kernel_name)
    if rec is None:
        return None
    return rec.get("dram_bytes_per_launch")


def cpu_baseline(prob, target_s=15.0, gpu=None, err_prob=None):
    """The oracle as it stands on this host: density (Newton, brute force over
    all N) + forces for a sample of sink particles; particle-steps/s.  With
    the GPU's t = 0 fields given, also the per-field error of the GPU path
    against the oracle (error_vs_oracle)."""
    import oracle
    from oracle import build as obuild
    obuild.build()
    p = oracle.Params(gamma=prob.gamma, alpha=prob.alpha, beta=prob.beta,
                      box_lo=prob.box_lo, box_hi=prob.box_hi, periodic=prob.periodic)
    rng = np.random.default_rng(0)

    def run(S):
        sinks = rng.choice(prob.n, size=S, replace=False)
        t0 = time.perf_counter()
        d = oracle.density_h(p, prob.pos, prob.m, prob.h0, sinks)
        h = np.array(prob.h0, dtype=np.float64)
        rho = np.ones(prob.n)
        om = np.ones(prob.n)
        h[sinks], rho[sinks], om[sinks] = d["h"], d["rho"], d["omega"]
        oracle.forces(p, prob.pos, prob.vel, prob.m, h, rho, om, prob.u, sinks)
        return time.perf_counter() - t0

    # calibrate on two sizes, then one run of about target_s seconds
    run(64)
    t = run(1024)
    S = int(min(prob.n, max(1024, 1024 * target_s / max(t, 1e-3))))
    t = run(S)
    cores = int(oracle.lib().orc_num_threads())
    out = {"value": S / t, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%d random sink particles of the t=0 state: Newton density (seeded from "
                     "the lattice h) and forces, each brute force over all %d particles in "
                     "FP64; %.1f s" % (S, prob.n, t)}
    err = error_vs_oracle(err_prob or prob, gpu, p) if gpu is not None else None
    return out, err


def gpu_fields(prob, params, dev):
    """One evaluation of a state on the GPU through the C ABI (build_cells,
    density_h seeded from prob.h0, forces) with the timed layout knobs;
    fields in input order."""
    import paper_2511_11425_gb300 as sph
    parts = sph.Particles.from_problem(prob, dev)
    ctx = sph.sph_create(params, prob.n)
    try:
        sph.sph_build_cells(ctx, parts)
        sph.sph_density_h(ctx, parts)
        sph.sph_forces(ctx, parts)
        g = parts.numpy()
    finally:
        sph.sph_destroy(ctx)
    order = np.argsort(g["id"], kind="stable")
    out = {k: v[order] for k, v in g.items()}
    out["a"] = np.stack([out["a0"], out["a1"], out["a2"]], 1)
    return out


def error_vs_oracle(prob, gpu, p):
    """Per-field error of the GPU's fields of a state against the FP64 oracle on
    sampled sinks (compact clusters round seeded centres and the blast
    centre).  The oracle solves h, rho and Omega by brute force over all N for
    every particle within 2.2 h_max of a sink, so the sinks' force sums see
    exact neighbour values.  h, rho, Omega: max relative error; a, du/dt and
    div v: max error over the field's max norm (the parity tolerances are
    1e-5 and 2e-4)."""
    import oracle
    rng = np.random.default_rng(5)
    centres = np.concatenate([rng.random((5, 3)), [[0.5, 0.5, 0.5]]])
    lo, hi = np.array(prob.box_lo), np.array(prob.box_hi)
    L = hi - lo
    per = np.array(prob.periodic, dtype=bool)

    def wrap(d):
        d = d.copy()
        d[:, per] -= L[per] * np.round(d[:, per] / L[per])
        return d
    sinks = []
    for c in centres:
        d = wrap(prob.pos - (lo + c * L))
        sinks.extend(np.argsort((d * d).sum(1))[:24])
    sinks = np.unique(np.array(sinks))
    R = 2.2 * float(np.max(prob.h0))
    keep = np.zeros(prob.n, dtype=bool)
    for s_ in sinks:
        d = wrap(prob.pos - prob.pos[s_])
        keep |= (d * d).sum(1) < R * R
    hood = np.nonzero(keep)[0]
    t0 = time.perf_counter()
    d = oracle.density_h(p, prob.pos, prob.m, prob.h0, hood)
    h = np.zeros(prob.n)
    rho = np.ones(prob.n)
    om = np.ones(prob.n)
    h[hood], rho[hood], om[hood] = d["h"], d["rho"], d["omega"]
    f = oracle.forces(p, prob.pos, prob.vel, prob.m, h, rho, om, prob.u, sinks)
    secs = time.perf_counter() - t0

    def rel(a, b):
        return float(np.max(np.abs(a - b) / np.abs(b)))

    def norm(a, b):
        return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))
    return {"h": rel(gpu["h"][sinks], h[sinks]), "rho": rel(gpu["rho"][sinks], rho[sinks]),
            "omega": rel(gpu["omega"][sinks], om[sinks]), "a": norm(gpu["a"][sinks], f["a"]),
            "dudt_h": norm(gpu["dudt_h"][sinks], f["dudt_h"]),
            "dudt_av": norm(gpu["dudt_av"][sinks], f["dudt_av"]),
            "divv": norm(gpu["divv"][sinks], f["divv"]),
            "tolerance": {"h_rho_omega_rel": 1e-5, "a_dudt_divv_max_norm": 2e-4},
            "sinks": int(len(sinks)), "neighbourhood": int(len(hood)),
            "oracle_s": round(secs, 1)}


def combine_ranks(ms, n_local, steps, world):
    """Whole-job timing of independent replicas: the slowest rank's timed
    milliseconds (every rank passed a barrier before its timed region) and
    the particle-steps of all ranks per second of that time."""
    tmax = float(ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = (torch.device("cuda", torch.cuda.current_device())
               if dist.get_backend() == "nccl" else torch.device("cpu"))
        t = torch.tensor([tmax], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tmax = float(t.item())
    return tmax, world * n_local * steps / (tmax / 1000.0)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    prob = _workload(0)
    import oracle
    from oracle import build as obuild
    obuild.build()
    p = oracle.Params(gamma=prob.gamma, alpha=prob.alpha, beta=prob.beta,
                      box_lo=prob.box_lo, box_hi=prob.box_hi, periodic=prob.periodic)
    rng = np.random.default_rng(1)
    S = 512

    def one_step():
        sinks = rng.choice(prob.n, size=S, replace=False)
        t0 = time.perf_counter()
        d = oracle.density_h(p, prob.pos, prob.m, prob.h0, sinks)
        h = np.array(prob.h0, dtype=np.float64)
        h[sinks] = d["h"]
        rho = np.ones(prob.n)
        om = np.ones(prob.n)
        rho[sinks], om[sinks] = d["rho"], d["omega"]
        oracle.forces(p, prob.pos, prob.vel, prob.m, h, rho, om, prob.u, sinks)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        one_step()
    tot = sum(one_step() for _ in range(args.steps))
    value = S * args.steps / tot
    cores = int(oracle.lib().orc_num_threads())
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(prob, {"sample_per_step": S}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: %d random sinks of the t=0 state, density "
                                       "Newton + forces, brute force over all particles" % S},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def forms_batch(dev, steps, warmup):
    """The batched form against the plain form on the 256-instance workload.

    plain          one context per problem, sph_step called for each in turn
    batched        one batch context: one launch per phase over all instances
    batched_graph  the batch step captured once as a CUDA graph and replayed
    All three advance every instance by the same number of steps from the same
    state; the per-instance step sizes they end with are compared (the batched
    forms compute the same pairs as the plain one)."""
    import torch
    import paper_2511_11425_gb300 as sph
    from paper_2511_11425_gb300 import inputs

    probs = inputs.batch()
    ntot = sum(q.n for q in probs)
    s = torch.cuda.Stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def timed(step, ctxs):
        l0 = sum(sph.sph_get_stats(c)["launches"] for c in ctxs)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        dp = fp = 0
        with torch.cuda.stream(s):
            for k in range(steps):
                flush.zero_()
                ev[k][0].record(s)
                step()
                ev[k][1].record(s)
                for c in ctxs:
                    st = sph.sph_get_stats(c)
                    dp += st["density_pairs"]
                    fp += st["force_pairs"]
            s.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        l1 = sum(sph.sph_get_stats(c)["launches"] for c in ctxs)
        return {"value": ntot * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                "launches_per_step": (l1 - l0) / steps,
                "pair_interactions_per_s": (dp + fp) / (ms * 1e-3)}

    out = {"workload": "256 independent Sod (gamma 1.4) and Sedov (gamma 5/3) instances, "
                       "particle counts log-uniform in [2k, 200k]",
           "instances": len(probs), "particles": ntot, "steps": steps, "warmup": warmup}
    sims = [sph.Simulation(q, device=dev) for q in probs]
    last = [0.0] * len(sims)

    def plain():
        for k, sim in enumerate(sims):
            last[k] = sph.sph_step(sim.ctx, sim.parts, 0.0, s)
    with torch.cuda.stream(s):
        for _ in range(warmup):
            plain()
    out["plain"] = timed(plain, [sim.ctx for sim in sims])
    dt_plain = np.array(last)
    for sim in sims:
        sim.close()
    del sims
    torch.cuda.empty_cache()

    b = sph.BatchSimulation(probs, device=dev)
    with torch.cuda.stream(s):
        for _ in range(warmup):
            sph.sph_step(b.ctx, b.parts, 0.0, s)
    out["batched"] = timed(lambda: sph.sph_step(b.ctx, b.parts, 0.0, s), [b.ctx])
    dt_b = np.array(sph.sph_batch_get_dt(b.ctx, b.ninst))
    b.close()
    del b
    torch.cuda.empty_cache()

    g = sph.BatchSimulation(probs, device=dev)
    with torch.cuda.stream(s):
        sph.sph_step(g.ctx, g.parts, 0.0, s)
        g.capture(s)
        for _ in range(warmup - 1):
            sph.sph_graph_launch(g.ctx, s)
    out["batched_graph"] = timed(lambda: sph.sph_graph_launch(g.ctx, s), [g.ctx])
    dt_g = np.array(sph.sph_batch_get_dt(g.ctx, g.ninst))
    g.close()
    del g
    torch.cuda.empty_cache()

    # the same with the layout knobs picked by the autotuner
    from paper_2511_11425_gb300 import autotune
    plist = [sph.Params.for_problem(q) for q in probs]
    parts, offs = sph.Particles.from_problems(probs, dev)
    tuner = autotune.Autotuner(os.path.join(tempfile.gettempdir(), "sph_autotune.json"), steps=2)
    plist = tuner.tune(parts, plist, offs, force=True)
    del parts
    g = sph.BatchSimulation(probs, plist, device=dev)
    with torch.cuda.stream(s):
        sph.sph_step(g.ctx, g.parts, 0.0, s)
        g.capture(s)
        for _ in range(warmup - 1):
            sph.sph_graph_launch(g.ctx, s)
    out["batched_graph_tuned"] = timed(lambda: sph.sph_graph_launch(g.ctx, s), [g.ctx])
    out["batched_graph_tuned"]["knobs"] = tuner.report["knobs"]
    out["batched_graph_tuned"]["tuning_trials"] = len(tuner.report["tried"])
    dt_t = np.array(sph.sph_batch_get_dt(g.ctx, g.ninst))
    g.close()
    del g
    torch.cuda.empty_cache()

    out["speedup_vs_plain"] = {
        "batched": out["batched"]["value"] / out["plain"]["value"],
        "batched_graph": out["batched_graph"]["value"] / out["plain"]["value"],
        "batched_graph_tuned": out["batched_graph_tuned"]["value"] / out["plain"]["value"]}
    out["max_rel_dt_diff_vs_plain"] = {
        "batched": float(np.max(np.abs(dt_b - dt_plain) / dt_plain)),
        "batched_graph": float(np.max(np.abs(dt_g - dt_plain) / dt_plain)),
        "batched_graph_tuned": float(np.max(np.abs(dt_t - dt_plain) / dt_plain))}
    return out


def forms_learned(dev, n_total=8_000_000, nrec=50, ncmp=200, tol=1e-5):
    """The learned seed against the continuity seed on the colliding-spheres
    workload: record `nrec` plain steps, train the network on the GPU, then
    run the same `ncmp` steps from the same state both ways (the first 50
    plain steps train, the next 200 are seeded)."""
    import torch
    import paper_2511_11425_gb300 as sph
    from paper_2511_11425_gb300 import inputs

    prob = inputs.collision(n_total=n_total)
    params = sph.Params.for_problem(prob, h_rel_tol=tol)
    s = torch.cuda.current_stream(dev)
    sim = sph.Simulation(prob, params, device=dev)
    ref = sph.Simulation(prob, params, device=dev)
    out = {"workload": "two colliding 1/r gas spheres (radii 1 and 0.5, Mach 3, impact "
                       "parameter 0.5), hydro only, open boundaries",
           "particles": prob.n, "h_rel_tol": tol, "record_steps": nrec, "compare_steps": ncmp}
    try:
        sim.step(0.0, s)
        sph.sph_mlp_record(sim.ctx, True, capacity=4 << 20,
                           stride=max(1, prob.n * nrec // (4 << 20)))
        for _ in range(nrec):
            dt = sim.step(0.0, s)
        sph.sph_mlp_record(sim.ctx, False)
        out["samples"] = sph.sph_mlp_samples(sim.ctx)
        sph.sph_mlp_set_weights(sim.ctx, inputs.mlp_init(3))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        l0, _ = sph.sph_mlp_train(sim.ctx, 2000, batch=8192, lr=2e-3, seed=1, stream=s)
        _, l1 = sph.sph_mlp_train(sim.ctx, 2000, batch=8192, lr=5e-4, seed=2, stream=s)
        out["train"] = {"adam_steps": 4000, "batch": 8192, "ms": 1e3 * (time.perf_counter() - t0),
                        "loss_first": l0, "loss_last": l1}
        for k, v in sim.parts.t.items():
            ref.parts.t[k].copy_(v)
        sph.sph_set_dt_old(ref.ctx, dt)
        sph.sph_mlp_set_seed_mode(sim.ctx, "mlp")
        for name, m in (("continuity_seed", ref), ("learned_seed", sim)):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(ncmp)]
            it = kd = 0.0
            pairs = 0
            for k in range(ncmp):
                ev[k][0].record(s)
                sph.sph_step(m.ctx, m.parts, 0.0, s)
                ev[k][1].record(s)
                st = sph.sph_get_stats(m.ctx)
                kd += st["ms_density_kernel"]
                pairs += st["density_pairs"]
                it += float(m.parts.t["iters"].float().mean())
            torch.cuda.synchronize(dev)
            ms = sum(a.elapsed_time(b) for a, b in ev)
            out[name] = {"ms_per_step": ms / ncmp, "density_kernel_ms_per_step": kd / ncmp,
                         "newton_passes_per_particle": it / ncmp,
                         "density_pair_evaluations_per_step": pairs / ncmp}
        a = ref.parts.numpy()
        b = sim.parts.numpy()
        oa = np.argsort(a["id"])
        ob = np.argsort(b["id"])

        def rel(f):
            return float(np.max(np.abs(b[f][ob].astype(np.float64) /
                                       a[f][oa].astype(np.float64) - 1.0)))
        acc_a = np.stack([a["a%d" % i][oa] for i in range(3)], 1).astype(np.float64)
        acc_b = np.stack([b["a%d" % i][ob] for i in range(3)], 1).astype(np.float64)
        out["field_error_vs_continuity_seed"] = {
            "h_max_rel": rel("h"), "rho_max_rel": rel("rho"), "u_max_rel": rel("u"),
            "a_max_over_max_norm": float(np.max(np.abs(acc_b - acc_a)) / np.max(np.abs(acc_a)))}
        out["passes_saved"] = 1.0 - (out["learned_seed"]["newton_passes_per_particle"] /
                                     out["continuity_seed"]["newton_passes_per_particle"])
        out["step_speedup"] = (out["continuity_seed"]["ms_per_step"] /
                               out["learned_seed"]["ms_per_step"])
    finally:
        sim.close()
        ref.close()
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2511_11425_gb300 as sph

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    sph.lib()
    prob = _workload(rank)
    params = sph.Params.for_problem(prob)
    layout = {"autotuned": False}
    if args.layout:
        from paper_2511_11425_gb300 import autotune
        knobs = {}
        for item in args.layout.split(","):
            k, v = item.split("=")
            knobs[k] = v if k == "curve" else (int(v) if k == "group_log" else float(v))
        params = autotune.with_knobs(params, knobs)
        layout = {"autotuned": False, "knobs": knobs}
    elif not args.no_tune:
        from paper_2511_11425_gb300 import autotune
        tuner = autotune.Autotuner(os.path.join(tempfile.gettempdir(), "sph_autotune.json"), steps=3)
        params = tuner.tune(sph.Particles.from_problem(prob, dev), params, force=True)
        layout = {"autotuned": True, "knobs": tuner.report["knobs"],
                  "trials": len(tuner.report["tried"])}
    sim = sph.Simulation(prob, params, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

    # steady state = replays of the captured step (build, density with its
    # re-walk rounds, forces, kick-drift-kick, conserved totals); the first
    # warm-up step runs plainly so the captured state is a stepped one
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        sph.sph_step(sim.ctx, sim.parts, 0.0, s)
        sph.sph_graph_capture(sim.ctx, sim.parts, 0.0, s)
        for _ in range(max(args.warmup - 1, 0)):
            sph.sph_graph_launch(sim.ctx, s)

    def step():
        return sph.sph_graph_launch(sim.ctx, s)

    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    st0 = sph.sph_get_stats(sim.ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kd = kf = 0.0
    dpairs = fpairs = fav = dcand = fcand = 0
    phase = {k: 0.0 for k in ("ms_build", "ms_walk", "ms_density_kernel", "ms_density",
                              "ms_force_kernel", "ms_forces")}
    t_sim = 0.0
    with ClockSampler(local_rank) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(s):
                flush.zero_()
            ev[k][0].record(s)
            t_sim += step()
            ev[k][1].record(s)
            st = sph.sph_get_stats(sim.ctx)
            kd += st["ms_density_kernel"]
            kf += st["ms_force_kernel"]
            for key in phase:
                phase[key] += st[key] / args.steps
            dpairs += st["density_pairs"]
            fpairs += st["force_pairs"]
            fav += st["force_av_pairs"]
            dcand += st["density_candidates"]
            fcand += st["force_candidates"]
        torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    st1 = sph.sph_get_stats(sim.ctx)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    tmax, value = combine_ranks(ms, prob.n, args.steps, world)
    launches = int(st1["launches"] - st0["launches"])

    # roofline of the dominant pair kernel
    flop_d = FLOPS_DENSITY_PAIR * dpairs
    flop_f = FLOPS_FORCE_PAIR * fpairs + FLOPS_FORCE_AV * fav
    rd = {"kernel": "k_density", "bound": "alu", "achieved": flop_d / (kd * 1e-3) / 1e12,
          "ms_per_launch": kd / args.steps}
    rf = {"kernel": "k_forces", "bound": "alu", "achieved": flop_f / (kf * 1e-3) / 1e12,
          "ms_per_launch": kf / args.steps}
    dom, other = (rd, rf) if kd >= kf else (rf, rd)
    dom_file = "sph_density.cu" if dom is rd else "sph_forces.cu"
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp32_peak_tflops(sms)
    fma_measured, _ = fma_probe(s)
    roof = {"bound": "alu", "achieved": dom["achieved"], "peak": peak,
            "unit": "TFLOP/s", "frac": dom["achieved"] / peak,
            "traffic": _traffic_for(dom_file, dom["kernel"]), "kernel": dom["kernel"],
            "peak_source": "derived: %d SMs (device properties) x 128 FP32 lanes x 2 flop x "
                           "2.07 GHz" % sms,
            "fp32_fma_measured_tflops": fma_measured,
            "ms_per_launch": dom["ms_per_launch"]}
    # the hardware view of the same kernel (ncu, committed summary): pipe
    # utilisation counts every issued instruction, rejected candidates included
    rec = _ncu_record(dom_file, dom["kernel"])
    if rec and "fma_pipe_active_pct" in rec:
        roof["ncu_pipes_active_pct"] = {"fma": rec["fma_pipe_active_pct"],
                                        "alu": rec["alu_pipe_active_pct"]}
    other_line = {**other, "frac": other["achieved"] / peak}

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        prob2 = _workload(rank)
        host = sph.Particles.from_problem(prob2, "cpu", pin=True)
        ctx2 = sph.sph_create(params, prob2.n)
        try:
            # one plain step, then the step recorded as a graph on the
            # context's device buffers (replayed by every later call)
            sph.sph_step_host(ctx2, host, 0.0, s)
            sph.sph_step_host_capture(ctx2, host, 0.0, s)
            for _ in range(max(args.warmup - 1, 2)):
                sph.sph_step_host(ctx2, host, 0.0, s)
            tt = 0.0
            hb = db = 0
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                _, hbi, dbi = sph.sph_step_host(ctx2, host, 0.0, s)
                tt += time.perf_counter() - t0
                hb += hbi
                db += dbi
            # bytes per step, averaged: a refitting step copies m and id back
            # only when a re-sort changed them
            hb = hb // args.steps
            db = db // args.steps
        finally:
            sph.sph_destroy(ctx2)
        e2e = {"value": world * prob2.n * args.steps / tt, "unit": UNIT,
               "h2d_bytes_per_step": hb, "d2h_bytes_per_step": db}

    totals = sph.sph_graph_totals(sim.ctx)
    stepped = None
    if world == 1 and not args.no_cpu_baseline:
        # the stepped state (in motion round the blast) for the error report
        import dataclasses
        g = sim.parts.numpy()
        o = np.argsort(g["id"], kind="stable")
        stepped = dataclasses.replace(
            prob, pos=np.stack([g["x0"], g["x1"], g["x2"]], 1)[o],
            vel=np.stack([g["v0"], g["v1"], g["v2"]], 1)[o], u=g["u"][o],
            h0=g["h"][o].astype(np.float64))
    sim.close()
    forms = None
    if world == 1 and not args.no_forms:
        forms = {"batch": forms_batch(dev, max(2, min(args.steps, 5)), max(args.warmup, 3))}
        torch.cuda.empty_cache()
        forms["learned"] = forms_learned(dev)
        torch.cuda.empty_cache()
    cpu = err = None
    if world == 1 and not args.no_cpu_baseline:
        cpu, err = cpu_baseline(prob, gpu=gpu_fields(stepped, params, dev), err_prob=stepped)
        err["state"] = ("the state after the %d warm-up and %d timed steps, evaluated with "
                        "the timed layout knobs" % (args.warmup, args.steps))
    if rank == 0:
        secs = tmax / 1000.0
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": _config(prob, {"sim_time_covered": t_sim, "layout": layout,
                                         "step": "replay of the captured step (CUDA graph) "
                                                 "incl. conserved totals",
                                         "parallelism": "replicas" if world > 1 else "single"}),
                "conserved_after": {"mass": totals[0], "momentum": totals[1:4],
                                    "energy": totals[7] + totals[8]},
                "pair_interactions_per_s": {
                    "density": world * dpairs / secs, "force": world * fpairs / secs,
                    "total": world * (dpairs + fpairs) / secs},
                "candidates_per_useful_pair": {"density": dcand / max(dpairs, 1),
                                               "force": fcand / max(fpairs, 1)},
                "phase_ms_per_step": {
                    "build": phase["ms_build"],
                    "density_walk_newton_refit": phase["ms_density"],
                    "of_which_density_kernel": phase["ms_density_kernel"],
                    "forces_predict_walk_pairs_finalize_kdk_totals": phase["ms_forces"],
                    "of_which_force_kernel": phase["ms_force_kernel"],
                    "walks": phase["ms_walk"]},
                "roofline": roof, "roofline_other": other_line, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary(), "cpu_baseline": cpu,
                "error_vs_oracle": err,
                "forms": forms, "impl": "ours"}
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--layout", default="",
                    help="fixed layout knobs instead of tuning, e.g. curve=morton,bucket_cell=3")
    ap.add_argument("--no-tune", action="store_true",
                    help="run the default layout knobs instead of autotuning them first")
    ap.add_argument("--workload", default="sedov64", choices=sorted(WORKLOADS),
                    help="the timed problem: the Sedov-Taylor blast on 64^3 particles "
                         "(default) or the Kelvin-Helmholtz shear layer on 128^3")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the plain / batched / graph comparison on 256 instances")
    args = ap.parse_args(argv)
    _WORKLOAD[0] = args.workload
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
        try:
            return run_ours(args, rank, world, local_rank)
        finally:
            dist.destroy_process_group()
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
