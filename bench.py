"""Benchmark of the SPH hot path on GB300 (one JSON line on stdout).

Workload (default): the Kelvin-Helmholtz shear layer (Sec. 3.8 setting) on
a 128^3 = 2,097,152-particle jittered periodic lattice, Wendland C2 with 64
neighbours, alpha = 1, beta = 2, gamma = 5/3, mixed precision, autotuned
layout, starting at t = 0.  One step = sph_step: curve sort + bounds tree,
density/h Newton pass, force pass, kick-drift-kick with the Courant step
(every row of the hot path), plus the conserved-totals reduction.
--workload sedov64 times the Sedov-Taylor blast (Sec. 3.3) on 64^3 instead.

  value       particle-steps/s with the state resident in HBM; each timed step
              is one replay of the captured step (CUDA graph, conserved totals
              included) bracketed by CUDA events on its stream, and a 256 MiB
              buffer is written between steps so no step starts with a warm L2
  e2e         the same metric through sph_step_host (replaying the step that
              sph_step_host_capture recorded): the step's input arrays copied
              from pinned host memory, stepped, and every array copied back,
              all inside the timed region
  roofline    the dominant pair kernel against the FP32 pipe peak
              (SMs x 128 lanes x 2 flop x 2.07 GHz), algorithmic flops only
  roofline_hbm the memory-bound phases (sort, permute, buckets, predictor,
              finalize, kick-drift-kick, totals): algorithmic bytes per launch
              over the CUDA-event time per launch of a profiled pass, against
              the measured HBM copy bandwidth
  cpu_baseline the FP64 oracle on a bounded sample of the same state
  error_vs_oracle  per-field error of the GPU path against the oracle on
              sampled sinks of the stepped state (the 'stated error' of the
              metric), computed in the oracle's leg
  forms       the mixed-precision form against the plain FP64 form (Sedov
              64^3 to t = 0.05, KH 128^3), the batched form, the learned seed,
              and learned + mixed + batched against the plain form

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
# the planning estimate of the same work (about 30 flops per density pair per
# pass, about 100 per unique force pair), reported beside the tally
FLOPS_DENSITY_PAIR_EST = 30
FLOPS_FORCE_PAIR_EST = 100
METRIC = "SPH particle-steps/s"
UNIT = "particle-steps/s"


WORKLOADS = {
    "sedov64": "sedov_taylor_64^3 (262,144 particles, periodic unit box, t from 0)",
    "kh128": "kelvin_helmholtz_128^3 (2,097,152 particles, periodic unit box, t from 0)",
    "kh96": "kelvin_helmholtz_96^3 (884,736 particles, periodic unit box, t from 0; the "
            "size of the profiler captures)",
}
_WORKLOAD = ["kh128"]  # set from --workload
HBM_PEAK_GBS_FALLBACK = 6800.0


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json,
    driver-written), else the recipe's fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), \
            "measured"
    except (OSError, ValueError, KeyError):
        return HBM_PEAK_GBS_FALLBACK, "fallback"


# Algorithmic bytes per particle of the memory-bound phases (each array read
# or written once; FP64 x, v, u = 56 B, FP32 per-particle fields 4 B each):
#  keys      x (24) + instance (2) read, key (8) + index (4) written       = 38
#  sort      per 8-bit pass: keys read by the histogram (8), keys and
#            indices read and written by the scatter (24)                 = 32 x passes
#  permute   gather: index (4) + 111 B of particle arrays read, 111 written
#            to scratch; copy-back: 111 read, 111 written                 = 448
#  layout    keys, h, instance read twice (scan and apply)                = 28
#  buckets   x, m, h read (32), FP32 relative position + m (16) and
#            fixed-point position (16) written                            = 64
#  predict   v, u, a, du/dt, h, rho, Omega, relative position, instance
#            read (82), force records, accumulators written (80)          = 162
#  finalize  accumulators, records read (50), a, du/dt, div v, dt_i (28)  = 78
#  kdk       x, v, u, a, du/dt, div v, h, instance read (86); x, v, u, h
#            written (60)                                                 = 146
#  conserved x, v, u, m read                                              = 60
HBM_BYTES_PER_PARTICLE = {"keys": 38, "permute": 448, "layout": 28, "buckets": 64,
                          "predict": 162, "finalize": 78, "kdk": 146, "conserved": 60}
SORT_BYTES_PER_PASS = 32


def _workload(rank=0):
    from paper_2511_11425_gb300 import inputs
    if _WORKLOAD[0] in ("kh128", "kh96"):
        return inputs.kh(n=int(_WORKLOAD[0][2:]), seed=2511 + rank)
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
    1e-5 and 2e-4).  The max norm is the whole field's: the sample holds the
    particles where the GPU field is largest (_field_maxima), valued by the
    oracle."""
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
    sinks = np.unique(np.concatenate([np.array(sinks), _field_maxima(gpu)]))
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
            "max_norm": "over the sinks, which hold the %d particles of largest |value| of "
                        "each field" % FIELD_MAXIMA_PER_FIELD,
            "sinks": int(len(sinks)), "neighbourhood": int(len(hood)),
            "oracle_s": round(secs, 1)}


def phase_profile(prob, params, dev, steps=5, sort_passes=4):
    """Per-phase device time of plain steps (sph_set_profiling: CUDA events
    around each launch group) on a fresh copy of the workload, and the HBM
    roofline of the memory-bound phases: algorithmic bytes per launch (bytes
    per particle above x particles) over the measured time per launch."""
    import torch
    import paper_2511_11425_gb300 as sph
    import dataclasses
    peak, src = hbm_peak_gbs()
    # replays of the captured step as timed (conserved totals included),
    # recorded with profiling on; every step re-sorts, so the key, sort,
    # permute and layout phases are timed too
    sim = sph.Simulation(prob, dataclasses.replace(params, resort_period=1), device=dev)
    s = torch.cuda.Stream(dev)
    try:
        with torch.cuda.stream(s):
            for _ in range(3):
                sph.sph_step(sim.ctx, sim.parts, 0.0, s)
            sph.sph_set_profiling(sim.ctx, True)
            sph.sph_graph_capture(sim.ctx, sim.parts, 0.0, s)
            sph.sph_graph_launch(sim.ctx, s)
            sph.sph_set_profiling(sim.ctx, True)  # clears the totals so far
            for _ in range(steps):
                sph.sph_graph_launch(sim.ctx, s)
        torch.cuda.synchronize(dev)
        times = sph.sph_phase_times(sim.ctx)
    finally:
        sim.close()
    per = {k: {"ms_per_launch": ms / n, "launches_per_step": n / steps}
           for k, (ms, n) in times.items() if n > 0}
    bpp = dict(HBM_BYTES_PER_PARTICLE, sort=SORT_BYTES_PER_PASS * sort_passes)
    hbm = {}
    for k, b in bpp.items():
        if k not in per:
            continue
        nbytes = b * prob.n
        ms = per[k]["ms_per_launch"]
        gbs = nbytes / (ms * 1e-3) / 1e9
        hbm[k] = {"bound": "hbm", "bytes_per_particle": b, "bytes_per_launch": nbytes,
                  "ms_per_launch": ms, "achieved": gbs, "peak": peak, "unit": "GB/s",
                  "frac": gbs / peak}
    per_step = {k: ms / steps for k, (ms, n) in times.items() if n > 0}
    return {"phase_ms_per_launch": per, "phase_ms_per_step": per_step, "hbm": hbm,
            "peak_source": "%s copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" % src
            if src == "measured" else "profiling recipe fallback 6.8 TB/s"}


FIELD_MAXIMA_PER_FIELD = 4


def _field_maxima(*gpus):
    """Indices of the FIELD_MAXIMA_PER_FIELD particles with the largest |value|
    of a (largest component), du/dt|H, du/dt|Pi and div v in each GPU field
    set.  Added to an oracle sample they make its max norm the field's max
    norm: the oracle values them, so a mislocated maximum only lowers the
    norm (a stricter test)."""
    idx = []
    for g in gpus:
        for k in ("a", "dudt_h", "dudt_av", "divv"):
            v = np.abs(np.asarray(g[k], dtype=np.float64))
            mag = v.max(1) if v.ndim == 2 else v
            idx.extend(np.argsort(-mag, kind="stable")[:FIELD_MAXIMA_PER_FIELD].tolist())
    return np.array(idx, dtype=np.int64)


def _sampled_clusters(prob, centres, per):
    lo, hi = np.array(prob.box_lo), np.array(prob.box_hi)
    L = hi - lo
    perd = np.array(prob.periodic, dtype=bool)
    sinks = []
    for c in centres:
        d = prob.pos - np.asarray(c)
        d[:, perd] -= L[perd] * np.round(d[:, perd] / L[perd])
        sinks.extend(np.argsort((d * d).sum(1))[:per])
    return np.unique(np.array(sinks))


def _oracle_on(prob, sinks):
    """FP64 oracle density + forces of `sinks`, exact for them (every particle
    within 2.2 h_max of a sink solved by brute force over all N)."""
    import oracle
    p = oracle.Params(gamma=prob.gamma, alpha=prob.alpha, beta=prob.beta,
                      box_lo=prob.box_lo, box_hi=prob.box_hi, periodic=prob.periodic)
    lo, hi = np.array(prob.box_lo), np.array(prob.box_hi)
    L = hi - lo
    perd = np.array(prob.periodic, dtype=bool)
    R = 2.2 * float(np.max(prob.h0))
    keep = np.zeros(prob.n, dtype=bool)
    for s_ in sinks:
        d = prob.pos - prob.pos[s_]
        d[:, perd] -= L[perd] * np.round(d[:, perd] / L[perd])
        keep |= (d * d).sum(1) < R * R
    hood = np.nonzero(keep)[0]
    d = oracle.density_h(p, prob.pos, prob.m, prob.h0, hood)
    h = np.zeros(prob.n)
    rho = np.ones(prob.n)
    om = np.ones(prob.n)
    h[hood], rho[hood], om[hood] = d["h"], d["rho"], d["omega"]
    f = oracle.forces(p, prob.pos, prob.vel, prob.m, h, rho, om, prob.u, sinks)
    return {"h": h[sinks], "rho": rho[sinks], "omega": om[sinks], **f}


def _field_errors(g, o, sinks):
    def rel(a, b):
        return float(np.max(np.abs(a - b) / np.abs(b)))

    def norm(a, b):
        return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))
    return {"h": rel(g["h"][sinks], o["h"]), "rho": rel(g["rho"][sinks], o["rho"]),
            "omega": rel(g["omega"][sinks], o["omega"]), "a": norm(g["a"][sinks], o["a"]),
            "dudt_h": norm(g["dudt_h"][sinks], o["dudt_h"]),
            "dudt_av": norm(g["dudt_av"][sinks], o["dudt_av"]),
            "divv": norm(g["divv"][sinks], o["divv"])}


def forms_precision(dev, kh_steps=5):
    """The mixed-precision form against the plain FP64 form.

    Sedov-Taylor 64^3 from t = 0 to t = 0.05 under the method's own global
    step, both forms timed step by step (plain sph_step); at the end the
    shock radius and energy error of each against the similarity solution.
    Kelvin-Helmholtz 128^3: kh_steps timed steps of each form.  Accuracy:
    both forms evaluated on the t = 0 state of each problem against the FP64
    oracle on sampled sinks (at the shear interfaces and round the blast)."""
    import torch
    import paper_2511_11425_gb300 as sph
    from paper_2511_11425_gb300 import inputs
    from oracle.sedov import SedovSolution
    out = {}
    s = torch.cuda.current_stream(dev)

    def run(prob, mode, t_end=None, nsteps=None):
        params = sph.Params.for_problem(prob, precision=mode)
        sim = sph.Simulation(prob, params, device=dev)
        m64 = prob.m.astype(np.float32).astype(np.float64)
        E0 = float((m64 * (prob.u + 0.5 * (prob.vel ** 2).sum(1))).sum())
        ms, steps, dt = 0.0, 0, 0.0
        try:
            sim.step()  # first step (t = 0 evaluation) untimed
            steps += 1
            while (t_end is not None and sim.t < t_end) or (nsteps is not None and
                                                             steps < nsteps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                dt = sim.step(0.0, s)
                e1.record(s)
                e1.synchronize()
                ms += e0.elapsed_time(e1)
                steps += 1
            g = sim.parts.numpy()
        finally:
            sim.close()
        o = np.argsort(g["id"], kind="stable")
        v = np.stack([g["v%d" % k][o] for k in range(3)], 1)
        a = np.stack([g["a%d" % k][o] for k in range(3)], 1)
        vs = v - 0.5 * dt * a
        us = g["u"][o] - 0.5 * dt * (g["dudt_h"][o].astype(np.float64) + g["dudt_av"][o])
        E1 = float((m64 * (us + 0.5 * (vs ** 2).sum(1))).sum())
        x = np.stack([g["x%d" % k][o] for k in range(3)], 1)
        timed = steps - 1
        return {"particle_steps_per_s": prob.n * timed / (ms * 1e-3), "ms_per_step": ms / timed,
                "timed_steps": timed, "t_end": sim.t, "energy_rel_error": abs(E1 - E0) / E0,
                "x": x, "rho": g["rho"][o]}

    sed = inputs.sedov(n=64)
    sol = SedovSolution(sed.gamma)
    res = {}
    for mode in ("mixed", "fp64"):
        r = run(sed, mode, t_end=0.05)
        rr = np.linalg.norm(r.pop("x") - 0.5, axis=1)
        rho = r.pop("rho")
        edges = np.linspace(0.0, 0.5, 51)
        idx = np.digitize(rr, edges) - 1
        prof = np.array([rho[idx == k].mean() if np.any(idx == k) else 0.0 for k in range(50)])
        r["shock_radius_peak"] = float(0.5 * (edges[np.argmax(prof)] + edges[np.argmax(prof) + 1]))
        r["shock_radius_analytic"] = float(sol.shock_radius(r["t_end"]))
        res[mode] = r
        torch.cuda.empty_cache()
    res["speedup_mixed_over_fp64"] = (res["mixed"]["particle_steps_per_s"] /
                                      res["fp64"]["particle_steps_per_s"])
    out["sedov64_to_t0.05"] = res
    kh = inputs.kh(n=128)
    res = {}
    for mode in ("mixed", "fp64"):
        r = run(kh, mode, nsteps=kh_steps)
        r.pop("x")
        r.pop("rho")
        res[mode] = r
        torch.cuda.empty_cache()
    res["speedup_mixed_over_fp64"] = (res["mixed"]["particle_steps_per_s"] /
                                      res["fp64"]["particle_steps_per_s"])
    out["kh128"] = res
    # accuracy of both forms on the t = 0 states
    acc = {}
    for name, prob, centres in (
            ("sedov64", sed, [[0.5, 0.5, 0.5], [0.2, 0.7, 0.4]]),
            ("kh128", kh, [[0.3, 0.25, 0.6], [0.7, 0.75, 0.2], [0.5, 0.5, 0.5]])):
        gs = {mode: gpu_fields(prob, sph.Params.for_problem(prob, precision=mode), dev)
              for mode in ("mixed", "fp64")}
        sinks = np.unique(np.concatenate([_sampled_clusters(prob, centres, 16),
                                          _field_maxima(*gs.values())]))
        t0 = time.perf_counter()
        o = _oracle_on(prob, sinks)
        acc[name] = {"sinks": int(len(sinks)), "oracle_s": round(time.perf_counter() - t0, 1)}
        for mode in ("mixed", "fp64"):
            acc[name][mode] = _field_errors(gs[mode], o, sinks)
    acc["tolerance"] = {"h_rho_omega_rel": 1e-5, "a_dudt_divv_max_norm": 2e-4}
    out["error_vs_oracle_t0"] = acc
    return out


def forms_combined(dev, steps=3, warmup=3, nrec=12):
    """The learned-seed + mixed-precision + batched form against the plain
    form on the 256-instance workload: plain = one context per problem in
    the FP64 form with the continuity seed, each stepped by sph_step in turn;
    combined = one batch context in the mixed form, autotuned layout, the
    step captured as a CUDA graph, the h iteration seeded by the network
    trained on the batch's own first nrec steps.  Both start from the same
    state and run the same number of steps."""
    import torch
    import paper_2511_11425_gb300 as sph
    from paper_2511_11425_gb300 import autotune, inputs
    probs = inputs.batch()
    ntot = sum(q.n for q in probs)
    s = torch.cuda.Stream(dev)
    out = {"workload": "256 independent Sod and Sedov instances (batch workload)",
           "particles": ntot, "steps": steps}
    # plain form
    sims = [sph.Simulation(q, sph.Params.for_problem(q, precision="fp64"), device=dev)
            for q in probs]
    with torch.cuda.stream(s):
        for _ in range(warmup):
            for sim in sims:
                sph.sph_step(sim.ctx, sim.parts, 0.0, s)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            for sim in sims:
                sph.sph_step(sim.ctx, sim.parts, 0.0, s)
        e1.record(s)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    out["plain_fp64_per_problem"] = {"value": ntot * steps / (ms * 1e-3),
                                     "ms_per_step": ms / steps}
    for sim in sims:
        sim.close()
    del sims
    torch.cuda.empty_cache()
    # combined form
    plist = [sph.Params.for_problem(q) for q in probs]
    parts, offs = sph.Particles.from_problems(probs, dev)
    tuner = autotune.Autotuner(os.path.join(tempfile.gettempdir(), "sph_autotune.json"), steps=2)
    plist = tuner.tune(parts, plist, offs)
    del parts
    b = sph.BatchSimulation(probs, plist, device=dev)
    try:
        with torch.cuda.stream(s):
            sph.sph_step(b.ctx, b.parts, 0.0, s)
            sph.sph_mlp_record(b.ctx, True, capacity=2 << 20,
                               stride=max(1, ntot * nrec // (2 << 20)))
            for _ in range(nrec):
                sph.sph_step(b.ctx, b.parts, 0.0, s)
            sph.sph_mlp_record(b.ctx, False)
            sph.sph_mlp_set_weights(b.ctx, inputs.mlp_init(3))
            sph.sph_mlp_train(b.ctx, 1500, batch=8192, lr=2e-3, seed=1, stream=s)
            sph.sph_mlp_train(b.ctx, 1500, batch=8192, lr=5e-4, seed=2, stream=s)
            sph.sph_mlp_set_seed_mode(b.ctx, "mlp")
            sph.sph_step(b.ctx, b.parts, 0.0, s)
            b.capture(s)
            for _ in range(warmup - 1):
                sph.sph_graph_launch(b.ctx, s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(steps):
                sph.sph_graph_launch(b.ctx, s)
            e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    finally:
        b.close()
    out["learned_mixed_batched"] = {"value": ntot * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                                    "knobs": tuner.report["knobs"]}
    out["speedup"] = out["learned_mixed_batched"]["value"] / out["plain_fp64_per_problem"]["value"]
    # accuracy: both arithmetic forms on the t = 0 states of the smallest and
    # largest instance against the oracle
    sizes = np.array([q.n for q in probs])
    acc = {}
    for k in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        q = probs[k]
        lo, hi = np.array(q.box_lo), np.array(q.box_hi)
        c = [0.5 * (lo + hi), lo + 0.3 * (hi - lo)]
        gs = {mode: gpu_fields(q, sph.Params.for_problem(q, precision=mode), dev)
              for mode in ("mixed", "fp64")}
        sinks = np.unique(np.concatenate([_sampled_clusters(q, c, 12),
                                          _field_maxima(*gs.values())]))
        o = _oracle_on(q, sinks)
        acc["instance_%d_%s_%d" % (k, q.name, q.n)] = {
            mode: _field_errors(gs[mode], o, sinks) for mode in ("mixed", "fp64")}
    out["error_vs_oracle_t0"] = acc
    torch.cuda.empty_cache()
    return out


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


def forms_rungs(dev, R=6, nglobal=2):
    """Hierarchical steps (Sec. 2.3.6) on Sedov-Taylor 64^3: one global step
    dt0 = 2^R x 0.9 x the smallest step limit of the start, taken (a) as 2^R
    plain global steps of dt0 / 2^R, (b) with rungs, every substep solving
    every particle, (c) with rungs and FastGas.  Device time per dt0 after one
    untimed global step; the rung histogram at the end."""
    import torch
    import paper_2511_11425_gb300 as sph
    from paper_2511_11425_gb300 import inputs
    prob = inputs.sedov(n=64)
    params = sph.Params.for_problem(prob)
    sim = sph.Simulation(prob, params, device=dev)
    try:
        sph.sph_build_cells(sim.ctx, sim.parts)
        sph.sph_density_h(sim.ctx, sim.parts)
        sph.sph_forces(sim.ctx, sim.parts)
        dt_min = float(sim.parts.t["dt_i"].min().item())
    finally:
        sim.close()
    dt0 = 2 ** R * dt_min * 0.9
    s = torch.cuda.current_stream(dev)
    out = {"workload": "sedov_taylor_64^3 (262,144 particles) from t = 0", "max_rung": R,
           "dt0": dt0}

    def timed(run_one):
        run_one()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(nglobal):
            run_one()
        b.record(s)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / nglobal

    sim = sph.Simulation(prob, params, device=dev)
    try:
        out["global_steps_ms_per_dt0"] = timed(
            lambda: [sim.step(dt0 / 2 ** R) for _ in range(2 ** R)])
    finally:
        sim.close()
    for name, fg in (("rungs_full_ms_per_dt0", False), ("rungs_fastgas_ms_per_dt0", True)):
        sim = sph.Simulation(prob, params, device=dev)
        try:
            sph.sph_set_fastgas(sim.ctx, fg)
            out[name] = timed(lambda: sph.sph_step_rungs(sim.ctx, sim.parts, dt0, R))
            if fg:
                out["rung_histogram"] = np.bincount(sph.sph_get_rungs(sim.ctx, prob.n),
                                                    minlength=R + 1).tolist()
        finally:
            sim.close()
    out["fastgas_speedup_over_full_rungs"] = (out["rungs_full_ms_per_dt0"] /
                                              out["rungs_fastgas_ms_per_dt0"])
    out["fastgas_speedup_over_global_steps"] = (out["global_steps_ms_per_dt0"] /
                                                out["rungs_fastgas_ms_per_dt0"])
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
          "achieved_at_estimate": FLOPS_DENSITY_PAIR_EST * dpairs / (kd * 1e-3) / 1e12,
          "ms_per_launch": kd / args.steps}
    rf = {"kernel": "k_forces", "bound": "alu", "achieved": flop_f / (kf * 1e-3) / 1e12,
          "achieved_at_estimate": FLOPS_FORCE_PAIR_EST * fpairs / (kf * 1e-3) / 1e12,
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
            "frac_at_estimate": dom["achieved_at_estimate"] / peak,
            "flops_per_unit": ("26 per density pair per pass" if dom is rd else
                               "61 per force pair + 24 per viscous pair") +
                              " (tally); estimate 30 / 100",
            "ms_per_launch": dom["ms_per_launch"]}
    # the hardware view of the same kernel (ncu, committed summary): pipe
    # utilisation counts every issued instruction, rejected candidates included
    rec = _ncu_record(dom_file, dom["kernel"])
    if rec and "fma_pipe_active_pct" in rec:
        roof["ncu_pipes_active_pct"] = {"fma": rec["fma_pipe_active_pct"],
                                        "alu": rec["alu_pipe_active_pct"]}
    other_line = {**other, "frac": other["achieved"] / peak,
                  "frac_at_estimate": other["achieved_at_estimate"] / peak}
    profile = None
    if not args.no_profile:
        profile = phase_profile(prob, params, dev)

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
        todo = {"precision": lambda: forms_precision(dev),
                "batch": lambda: forms_batch(dev, max(2, min(args.steps, 5)),
                                             max(args.warmup, 3)),
                "learned": lambda: forms_learned(dev), "rungs": lambda: forms_rungs(dev),
                "combined": lambda: forms_combined(dev)}
        only = [f for f in args.forms.split(",") if f] if args.forms else list(todo)
        forms = {}
        for name in only:
            forms[name] = todo[name]()
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
                "roofline": roof, "roofline_other": other_line,
                "roofline_hbm": profile["hbm"] if profile else None,
                "phase_profile": ({"ms_per_step": profile["phase_ms_per_step"],
                                   "note": "replays of the captured step (totals included) "
                                           "that all re-sort",
                                   "hbm_peak": profile["peak_source"]} if profile else None),
                "e2e": e2e,
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
    ap.add_argument("--workload", default="kh128", choices=sorted(WORKLOADS),
                    help="the timed problem: the Kelvin-Helmholtz shear layer on 128^3 "
                         "particles (default), on 96^3 (profiler captures), or the "
                         "Sedov-Taylor blast on 64^3")
    ap.add_argument("--no-profile", action="store_true",
                    help="skip the per-phase timing pass (HBM roofline of the "
                         "memory-bound phases)")
    ap.add_argument("--forms", default="",
                    help="comma-separated subset of the forms to run (precision, batch, "
                         "learned, rungs, combined); default all")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the form comparisons (FP64 against mixed precision, "
                         "batched, learned seed, combined)")
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
