"""Autotuner for the layout knobs of the SPH step.

The step's cost depends on how particles are cut into warps and walks, not
only on the hardware: the space-filling curve, the buckets per walk group
(the paper's group size of Sec. 2.3.2), the largest key cell a bucket may
span (in units of h), the margin of the density lists (Sec. 2.3.3: lists
are built for a slightly larger kernel) and how often the particles are
re-sorted (between re-sorts the buckets' bounds are refitted).  None of
them changes the result beyond rounding; each changes the candidates per
useful pair, the walk work, the warp fill or the build work.  The tuner times whole steps of the caller's own state
(on a copy) for candidate settings, one knob at a time (coordinate
descent from the defaults), keeps the fastest, and caches the choice per
GPU and configuration class (size, instance count, boundaries, kernel,
neighbour number) in a JSON file.

    tuner = Autotuner()
    params = tuner.tune(parts, params)                 # one problem
    plist = tuner.tune(parts, plist, offsets)          # a batch
"""
from __future__ import annotations

import dataclasses
import json
import math
import os

SPACE = {
    "curve": ["hilbert", "morton"],
    "group_log": [3, 2],
    "bucket_cell": [3.0, 2.0, 4.0],
    "list_margin": [0.1, 0.05, 0.2],
    "resort_period": [1, 4, 8, 16],
}
ORDER = ("resort_period", "curve", "bucket_cell", "group_log", "list_margin")


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "paper_2511_11425_gb300", "autotune.json")


def config_class(n: int, params_list, device_name: str) -> str:
    """Cache key: GPU, particle count and instance count to the nearest power
    of two, boundaries, kernel and neighbour number of the first instance."""
    p = params_list[0]
    per = "".join("p" if x else "o" for x in p.periodic)
    return "%s|n2^%d|inst2^%d|%s|%s|nngb%g" % (
        device_name, round(math.log2(max(n, 1))), round(math.log2(max(len(params_list), 1))),
        per, p.kernel, p.n_ngb)


def with_knobs(params, knobs: dict):
    """params with the tuned knobs applied (the group bound follows the bucket
    bound: twice it, at least 6 h)."""
    kw = dict(knobs)
    if "bucket_cell" in kw:
        kw["group_cell"] = max(6.0, 2.0 * kw["bucket_cell"])
    return dataclasses.replace(params, **kw)


def coordinate_descent(measure, start: dict, space=SPACE, order=ORDER, rel_gain=0.02):
    """Minimise measure(knobs) one knob at a time from `start`; a change is
    kept only when it is faster by more than rel_gain.  Returns (best knobs,
    best time, list of (knobs, time) tried)."""
    cur = dict(start)
    best = measure(cur)
    tried = [(dict(cur), best)]
    for name in order:
        for v in space[name]:
            if v == cur[name]:
                continue
            cand = dict(cur)
            cand[name] = v
            t = measure(cand)
            tried.append((dict(cand), t))
            if t < best * (1.0 - rel_gain):
                cur, best = cand, t
    return cur, best, tried


class Autotuner:
    def __init__(self, cache_path: str | None = None, steps: int = 3, warmup: int = 1,
                 measure=None):
        self.cache_path = cache_path or default_cache_path()
        self.steps = steps
        self.warmup = warmup
        self._measure = measure     # measure(parts, params_list, offsets) -> ms per step
        self.report = None

    # ---- cache ---------------------------------------------------------------
    def _load(self) -> dict:
        try:
            with open(self.cache_path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}

    def _store(self, key: str, knobs: dict, ms: float):
        data = self._load()
        data[key] = {"knobs": knobs, "ms_per_step": ms}
        os.makedirs(os.path.dirname(os.path.abspath(self.cache_path)), exist_ok=True)
        tmp = self.cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    # ---- timing --------------------------------------------------------------
    def _time_steps(self, parts, params_list, offsets) -> float:
        """ms per step of the given settings on a copy of the particles."""
        import torch
        from . import (Particles, sph_batch_create, sph_create, sph_destroy, sph_step)
        dev = parts.t["x0"].device
        work = Particles(parts.n, dev)
        for k, v in parts.t.items():
            work.t[k].copy_(v)
        if offsets is None:
            ctx = sph_create(params_list[0], parts.n)
        else:
            ctx = sph_batch_create(params_list, offsets)
        s = torch.cuda.current_stream(dev)
        # whole re-sort periods, so every setting is timed on its own mix
        period = max(p.resort_period for p in params_list)
        steps = period * max(1, -(-self.steps // period))
        try:
            for _ in range(self.warmup):
                sph_step(ctx, work, 0.0, s)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            for _ in range(steps):
                sph_step(ctx, work, 0.0, s)
            b.record(s)
            b.synchronize()
            return a.elapsed_time(b) / steps
        finally:
            sph_destroy(ctx)

    def tune(self, parts, params, offsets=None, device_name=None, force=False):
        """Tuned Params (or list of Params for a batch, given offsets)."""
        single = not isinstance(params, (list, tuple))
        plist = [params] if single else list(params)
        if device_name is None:
            import torch
            device_name = torch.cuda.get_device_name(parts.t["x0"].device)
        key = config_class(parts.n, plist, device_name)
        cache = self._load()
        if key in cache and not force:
            knobs = cache[key]["knobs"]
            self.report = {"key": key, "cached": True, "knobs": knobs}
        else:
            measure = self._measure or self._time_steps
            start = {k: getattr(plist[0], k) for k in ORDER}

            def run(knobs):
                return measure(parts, [with_knobs(p, knobs) for p in plist], offsets)
            knobs, ms, tried = coordinate_descent(run, start)
            self._store(key, knobs, ms)
            self.report = {"key": key, "cached": False, "knobs": knobs, "ms_per_step": ms,
                           "tried": [{"knobs": k, "ms_per_step": t} for k, t in tried]}
        out = [with_knobs(p, knobs) for p in plist]
        return out[0] if single else out
