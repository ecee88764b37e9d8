"""GB300-native SPH hot path: Python binding of libsph (include/sph.h).

This module only marshals arguments: device arrays are torch tensors whose
data pointers go into the C structs, streams are passed as raw handles.
Every computation runs in the CUDA kernels of ``_libsph.so``.  There is no
fallback: if the library is missing or cannot be loaded, every call raises.

Functions carry the C names (``sph_create``, ``sph_build_cells``,
``sph_density_h``, ``sph_density_at``, ``sph_forces``, ``sph_kdk_step``,
``sph_step``, ``sph_step_host``, ``sph_reduce_conserved``, ``sph_set_dt_old``,
``sph_get_stats``, ``sph_last_error``, ``sph_version``, ``sph_destroy``) and
raise ``SphError`` on a non-OK status.  ``Params`` and ``Particles`` build the
C structs; ``Simulation`` strings the calls together for one problem.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_libsph.so")

STATUS = {0: "SPH_OK", 1: "SPH_ERR_ARG", 2: "SPH_ERR_CUDA", 3: "SPH_ERR_CAPACITY",
          4: "SPH_ERR_NOCONV", 5: "SPH_ERR_NONFINITE", 7: "SPH_ERR_STATE"}
KERNELS = {"wc2": 0, "wc4": 1, "wc6": 2, "m4": 3}
ENERGY = {"pdv": 0, "isentropic": 1}
CURVES = {"hilbert": 0, "morton": 1}
PRECISIONS = {"mixed": 0, "fp64": 1}
DENSITY_MODES = {"summed": 0, "evolved": 1}
EXPORTS = ("sph_create", "sph_destroy", "sph_build_cells", "sph_density_h", "sph_density_at",
           "sph_forces", "sph_kdk_step", "sph_step", "sph_step_host", "sph_reduce_conserved",
           "sph_set_dt_old", "sph_get_stats", "sph_last_error", "sph_version",
           "sph_reduce_conserved_noalloc", "sph_batch_create", "sph_batch_get_dt",
           "sph_graph_capture", "sph_graph_launch", "sph_graph_totals", "sph_mlp_set_weights", "sph_mlp_get_weights",
           "sph_mlp_set_seed_mode", "sph_mlp_record", "sph_mlp_samples", "sph_mlp_get_samples",
           "sph_mlp_load_samples", "sph_bucket_layout", "sph_set_list_arena", "sph_set_profiling",
           "sph_step_rungs", "sph_get_rungs", "sph_set_fastgas",
           "sph_mlp_train", "sph_mlp_grad", "sph_mlp_infer")
MLP_NPARAM = 1249
SEED_MODES = {"analytic": 0, "mlp": 1}


class SphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class c_params(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("energy_mode", C.c_int32), ("n_ngb", C.c_double),
                ("gamma", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
                ("eps_av", C.c_double), ("eta_courant", C.c_double), ("eta_acc", C.c_double),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
                ("periodic", C.c_int32 * 3), ("max_newton", C.c_int32),
                ("h_rel_tol", C.c_double), ("list_margin", C.c_double),
                ("curve", C.c_int32), ("group_log", C.c_int32),
                ("bucket_cell", C.c_double), ("group_cell", C.c_double),
                ("resort_period", C.c_int32), ("precision", C.c_int32),
                ("density_mode", C.c_int32), ("interface_correction", C.c_int32),
                ("ic_alpha", C.c_double), ("r_gas", C.c_double * 4)]


class c_particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p * 3), ("v", C.c_void_p * 3),
                ("u", C.c_void_p), ("m", C.c_void_p), ("h", C.c_void_p), ("rho", C.c_void_p),
                ("omega", C.c_void_p), ("a", C.c_void_p * 3), ("dudt_h", C.c_void_p),
                ("dudt_av", C.c_void_p), ("divv", C.c_void_p), ("dt_i", C.c_void_p),
                ("nngb", C.c_void_p), ("iters", C.c_void_p), ("id", C.c_void_p),
                ("mat", C.c_void_p)]


class c_stats(C.Structure):
    _fields_ = [("density_pairs", C.c_uint64), ("force_pairs", C.c_uint64),
                ("density_candidates", C.c_uint64), ("force_candidates", C.c_uint64),
                ("max_newton_iters", C.c_int32), ("relists", C.c_int32),
                ("list_entries_density", C.c_int64), ("list_entries_force", C.c_int64),
                ("dt_old", C.c_double), ("ms_build", C.c_float), ("ms_density", C.c_float),
                ("ms_forces", C.c_float), ("ms_kdk", C.c_float), ("ms_walk", C.c_float),
                ("ms_density_kernel", C.c_float), ("ms_force_kernel", C.c_float),
                ("pad_", C.c_int32), ("force_av_pairs", C.c_uint64), ("launches", C.c_uint64),
                ("phase_ms", C.c_double * 16), ("phase_launches", C.c_uint64 * 16)]


_lib = None


def lib():
    """Load _libsph.so (build it first with __graft_entry__.build() or build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsph is not built (%s missing); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
        L.sph_create.argtypes = [C.POINTER(c_params), i64, C.POINTER(vp)]
        L.sph_destroy.argtypes = [vp]
        L.sph_destroy.restype = None
        pp = C.POINTER(c_particles)
        L.sph_build_cells.argtypes = [vp, pp, vp]
        L.sph_density_h.argtypes = [vp, pp, vp, vp]
        L.sph_density_at.argtypes = [vp, pp, vp, i64, vp, vp, vp]
        L.sph_forces.argtypes = [vp, pp, vp]
        L.sph_kdk_step.argtypes = [vp, pp, dbl, C.POINTER(dbl), vp]
        L.sph_step.argtypes = [vp, pp, dbl, C.POINTER(dbl), vp]
        L.sph_step_host.argtypes = [vp, pp, dbl, C.POINTER(dbl), C.POINTER(i64),
                                    C.POINTER(i64), vp]
        L.sph_reduce_conserved.argtypes = [vp, pp, C.POINTER(dbl), vp]
        L.sph_reduce_conserved_noalloc.argtypes = [pp, vp, vp]
        L.sph_batch_create.argtypes = [C.POINTER(c_params), C.c_int32, C.POINTER(i64),
                                       C.POINTER(vp)]
        L.sph_batch_get_dt.argtypes = [vp, C.POINTER(dbl)]
        L.sph_graph_capture.argtypes = [vp, pp, dbl, vp]
        L.sph_step_host_capture.argtypes = [vp, pp, dbl, vp]
        L.sph_graph_launch.argtypes = [vp, C.POINTER(dbl), vp]
        L.sph_graph_totals.argtypes = [vp, C.POINTER(dbl)]
        L.sph_set_dt_old.argtypes = [vp, dbl]
        L.sph_set_list_arena.argtypes = [vp, i64]
        L.sph_set_profiling.argtypes = [vp, C.c_int32]
        L.sph_step_rungs.argtypes = [vp, pp, dbl, C.c_int32, vp]
        L.sph_get_rungs.argtypes = [vp, vp, i64]
        L.sph_set_fastgas.argtypes = [vp, C.c_int32]
        fp = C.POINTER(C.c_float)
        L.sph_mlp_set_weights.argtypes = [vp, fp, i64]
        L.sph_mlp_get_weights.argtypes = [vp, fp, i64]
        L.sph_mlp_set_seed_mode.argtypes = [vp, C.c_int32]
        L.sph_mlp_record.argtypes = [vp, C.c_int32, i64, C.c_int32]
        L.sph_mlp_samples.argtypes = [vp, C.POINTER(i64)]
        L.sph_mlp_get_samples.argtypes = [vp, fp, fp, i64]
        L.sph_mlp_load_samples.argtypes = [vp, vp, vp, i64, vp]
        L.sph_mlp_train.argtypes = [vp, C.c_int32, C.c_int32, dbl, C.c_uint64, C.POINTER(dbl),
                                    C.POINTER(dbl), vp]
        L.sph_mlp_grad.argtypes = [vp, vp, vp, i64, fp, C.POINTER(dbl), vp]
        L.sph_mlp_infer.argtypes = [vp, vp, i64, vp, vp]
        L.sph_bucket_layout.argtypes = [vp, C.POINTER(C.c_int32), i64, C.POINTER(i64)]
        L.sph_get_stats.argtypes = [vp, C.POINTER(c_stats)]
        L.sph_last_error.argtypes = [vp]
        L.sph_last_error.restype = C.c_char_p
        L.sph_version.argtypes = []
        L.sph_version.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("sph_destroy", "sph_last_error", "sph_version"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(ctx, rc):
    if rc != 0:
        msg = lib().sph_last_error(ctx).decode() if ctx else ""
        raise SphError(rc, msg)


def _stream(stream):
    if stream is None:
        return None
    return C.c_void_p(getattr(stream, "cuda_stream", stream))


@dataclasses.dataclass
class Params:
    """Python mirror of sph_params (defaults follow the paper's settings)."""
    kernel: str = "wc2"
    energy: str = "pdv"
    n_ngb: float = 64.0
    gamma: float = 5.0 / 3.0
    alpha: float = 1.0
    beta: float = 2.0
    eps_av: float = 0.01
    eta_courant: float = 0.15
    eta_acc: float = 0.2
    box_lo: tuple = (0.0, 0.0, 0.0)
    box_hi: tuple = (1.0, 1.0, 1.0)
    periodic: tuple = (1, 1, 1)
    max_newton: int = 64
    h_rel_tol: float = 1e-6
    list_margin: float = 0.1
    curve: str = "hilbert"
    group_log: int = 3
    bucket_cell: float = 3.0
    group_cell: float = 6.0
    resort_period: int = 1
    precision: str = "mixed"
    density: str = "summed"
    interface_correction: bool = False
    ic_alpha: float = 0.0
    r_gas: tuple = (1.0, 1.0, 1.0, 1.0)

    def c(self) -> c_params:
        p = c_params()
        p.kernel = KERNELS[self.kernel]
        p.energy_mode = ENERGY[self.energy]
        for f in ("n_ngb", "gamma", "alpha", "beta", "eps_av", "eta_courant", "eta_acc",
                  "h_rel_tol", "list_margin", "bucket_cell", "group_cell"):
            setattr(p, f, float(getattr(self, f)))
        p.max_newton = int(self.max_newton)
        p.curve = CURVES[self.curve]
        p.group_log = int(self.group_log)
        p.resort_period = int(self.resort_period)
        p.precision = PRECISIONS[self.precision]
        p.density_mode = DENSITY_MODES[self.density]
        p.interface_correction = 1 if self.interface_correction else 0
        p.ic_alpha = float(self.ic_alpha)
        for k in range(4):
            p.r_gas[k] = float(self.r_gas[k])
        for a in range(3):
            p.box_lo[a] = float(self.box_lo[a])
            p.box_hi[a] = float(self.box_hi[a])
            p.periodic[a] = int(bool(self.periodic[a]))
        return p

    @classmethod
    def for_problem(cls, prob, **kw):
        d = dict(kernel=prob.kernel, n_ngb=prob.n_ngb, gamma=prob.gamma, alpha=prob.alpha,
                 beta=prob.beta, box_lo=tuple(prob.box_lo), box_hi=tuple(prob.box_hi),
                 periodic=tuple(prob.periodic))
        d.update(kw)
        return cls(**d)


class Particles:
    """SoA particle state as torch tensors on one device, plus the C struct."""

    FIELDS64 = ("x0", "x1", "x2", "v0", "v1", "v2", "u")
    FIELDS32 = ("m", "h", "rho", "omega", "a0", "a1", "a2", "dudt_h", "dudt_av", "divv", "dt_i")

    def __init__(self, n, device="cuda", pin=False):
        import torch
        self.n = int(n)
        self.device = torch.device(device)
        kw = dict(device=self.device)
        if pin and self.device.type == "cpu":
            kw["pin_memory"] = True
        self.t = {}
        for f in self.FIELDS64:
            self.t[f] = torch.zeros(self.n, dtype=torch.float64, **kw)
        for f in self.FIELDS32:
            self.t[f] = torch.zeros(self.n, dtype=torch.float32, **kw)
        self.t["nngb"] = torch.zeros(self.n, dtype=torch.int16, **kw)
        self.t["iters"] = torch.zeros(self.n, dtype=torch.uint8, **kw)
        self.t["id"] = torch.arange(self.n, dtype=torch.int64, **kw)
        self.t["mat"] = torch.zeros(self.n, dtype=torch.uint8, **kw)

    @classmethod
    def from_problem(cls, prob, device="cuda", pin=False):
        import torch
        p = cls(prob.n, device, pin)
        for a in range(3):
            p.t["x%d" % a].copy_(torch.from_numpy(prob.pos[:, a].copy()))
            p.t["v%d" % a].copy_(torch.from_numpy(prob.vel[:, a].copy()))
        p.t["u"].copy_(torch.from_numpy(prob.u.copy()))
        p.t["m"].copy_(torch.from_numpy(prob.m.astype("float32")))
        p.t["h"].copy_(torch.from_numpy(prob.h0.astype("float32")))
        if "mat" in prob.extra:
            p.t["mat"].copy_(torch.from_numpy(prob.extra["mat"].astype("uint8")))
        return p

    @classmethod
    def from_problems(cls, probs, device="cuda", pin=False):
        """Concatenation of several problems (the layout of a batch context);
        returns (particles, offsets) with offsets[k]:offsets[k+1] = problem k."""
        import numpy as np
        import torch
        offs = np.cumsum([0] + [q.n for q in probs]).astype(np.int64)
        p = cls(int(offs[-1]), device, pin)

        def cat(get, dtype):
            return torch.from_numpy(np.concatenate([get(q) for q in probs]).astype(dtype))
        for a in range(3):
            p.t["x%d" % a].copy_(cat(lambda q: q.pos[:, a], "float64"))
            p.t["v%d" % a].copy_(cat(lambda q: q.vel[:, a], "float64"))
        p.t["u"].copy_(cat(lambda q: q.u, "float64"))
        p.t["m"].copy_(cat(lambda q: q.m, "float32"))
        p.t["h"].copy_(cat(lambda q: q.h0, "float32"))
        return p, offs

    def c(self) -> c_particles:
        s = c_particles()
        t = self.t
        s.n = self.n
        for a in range(3):
            s.x[a] = t["x%d" % a].data_ptr()
            s.v[a] = t["v%d" % a].data_ptr()
            s.a[a] = t["a%d" % a].data_ptr()
        for f in ("u", "m", "h", "rho", "omega", "dudt_h", "dudt_av", "divv", "dt_i", "nngb",
                  "iters", "id", "mat"):
            setattr(s, f, t[f].data_ptr())
        return s

    def pos(self):
        import torch
        return torch.stack([self.t["x0"], self.t["x1"], self.t["x2"]], 1)

    def vel(self):
        import torch
        return torch.stack([self.t["v0"], self.t["v1"], self.t["v2"]], 1)

    def acc(self):
        import torch
        return torch.stack([self.t["a0"], self.t["a1"], self.t["a2"]], 1)

    def numpy(self):
        """Host copy of every array, in the current (curve) order."""
        return {k: v.detach().cpu().numpy() for k, v in self.t.items()}


# ---- C-ABI calls, same names -------------------------------------------------
def sph_version() -> str:
    return lib().sph_version().decode()


def sph_create(params: Params, capacity: int):
    ctx = C.c_void_p()
    cp = params.c()
    rc = lib().sph_create(C.byref(cp), int(capacity), C.byref(ctx))
    _check(None, rc)
    return ctx


def sph_batch_create(params_list, offsets):
    """Context for independent problems: params_list[k] governs particles
    offsets[k]:offsets[k+1] of one concatenated Particles set."""
    n = len(params_list)
    cps = (c_params * n)(*[p.c() for p in params_list])
    offs = (C.c_int64 * (n + 1))(*[int(o) for o in offsets])
    ctx = C.c_void_p()
    rc = lib().sph_batch_create(cps, n, offs, C.byref(ctx))
    _check(None, rc)
    ctx.ninst = n
    return ctx


def sph_batch_get_dt(ctx, ninst):
    out = (C.c_double * ninst)()
    _check(ctx, lib().sph_batch_get_dt(ctx, out))
    return list(out)


def sph_graph_capture(ctx, parts: Particles, dt_fixed=0.0, stream=None):
    s = parts.c()
    _check(ctx, lib().sph_graph_capture(ctx, C.byref(s), float(dt_fixed), _stream(stream)))


def sph_graph_launch(ctx, stream=None) -> float:
    dt = C.c_double()
    _check(ctx, lib().sph_graph_launch(ctx, C.byref(dt), _stream(stream)))
    return dt.value


def sph_graph_totals(ctx, ninst=None):
    """Conserved totals after the last graph replay (9 per instance)."""
    k = ninst or getattr(ctx, "ninst", 1)
    out = (C.c_double * (9 * k))()
    _check(ctx, lib().sph_graph_totals(ctx, out))
    return list(out)


def sph_destroy(ctx):
    lib().sph_destroy(ctx)


def sph_build_cells(ctx, parts: Particles, stream=None):
    s = parts.c()
    _check(ctx, lib().sph_build_cells(ctx, C.byref(s), _stream(stream)))


def sph_density_h(ctx, parts: Particles, h_seed=None, stream=None):
    s = parts.c()
    hs = None if h_seed is None else C.c_void_p(h_seed.data_ptr())
    _check(ctx, lib().sph_density_h(ctx, C.byref(s), hs, _stream(stream)))


def sph_density_at(ctx, parts: Particles, h, cap=0, count=None, ids=None, stream=None):
    s = parts.c()
    cnt = None if count is None else C.c_void_p(count.data_ptr())
    idp = None if ids is None else C.c_void_p(ids.data_ptr())
    _check(ctx, lib().sph_density_at(ctx, C.byref(s), C.c_void_p(h.data_ptr()), int(cap), cnt,
                                     idp, _stream(stream)))


def sph_forces(ctx, parts: Particles, stream=None):
    s = parts.c()
    _check(ctx, lib().sph_forces(ctx, C.byref(s), _stream(stream)))


def sph_kdk_step(ctx, parts: Particles, dt_fixed=0.0, stream=None) -> float:
    s = parts.c()
    dt = C.c_double()
    _check(ctx, lib().sph_kdk_step(ctx, C.byref(s), float(dt_fixed), C.byref(dt), _stream(stream)))
    return dt.value


def sph_step(ctx, parts: Particles, dt_fixed=0.0, stream=None) -> float:
    s = parts.c()
    dt = C.c_double()
    _check(ctx, lib().sph_step(ctx, C.byref(s), float(dt_fixed), C.byref(dt), _stream(stream)))
    return dt.value


def sph_step_host(ctx, host_parts: Particles, dt_fixed=0.0, stream=None):
    """One step on host (CPU tensor) arrays; returns (dt, h2d_bytes, d2h_bytes)."""
    s = host_parts.c()
    dt = C.c_double()
    hb = C.c_int64()
    db = C.c_int64()
    _check(ctx, lib().sph_step_host(ctx, C.byref(s), float(dt_fixed), C.byref(dt), C.byref(hb),
                                    C.byref(db), _stream(stream)))
    return dt.value, hb.value, db.value


def sph_step_host_capture(ctx, host_parts: Particles, dt_fixed=0.0, stream=None):
    """Record one step on the context's device copy of host arrays; later
    sph_step_host calls with this dt_fixed replay it."""
    s = host_parts.c()
    _check(ctx, lib().sph_step_host_capture(ctx, C.byref(s), float(dt_fixed), _stream(stream)))


def sph_reduce_conserved(ctx, parts: Particles, stream=None, ninst=None):
    """Totals [M, P, L, E_kin, E_int] (9 values; 9 per instance for a batch)."""
    s = parts.c()
    k = ninst or getattr(ctx, "ninst", 1)
    out = (C.c_double * (9 * k))()
    _check(ctx, lib().sph_reduce_conserved(ctx, C.byref(s), out, _stream(stream)))
    return list(out)


def sph_reduce_conserved_noalloc(parts: Particles, out, stream=None):
    """Totals into `out` (a device tensor of 9 float64) without any allocation.

    Only queues the work: synchronise the stream before reading `out`.
    Raises ValueError unless `out` is a contiguous float64 CUDA tensor of at
    least 9 elements on the current device (the kernel writes 9 doubles)."""
    _check_totals_out(out)
    s = parts.c()
    _check(None, lib().sph_reduce_conserved_noalloc(C.byref(s), C.c_void_p(out.data_ptr()),
                                                    _stream(stream)))


def _check_totals_out(out):
    import torch
    if not isinstance(out, torch.Tensor):
        raise ValueError("out must be a torch tensor")
    if not out.is_cuda:
        raise ValueError("out must be a CUDA tensor")
    if out.dtype != torch.float64:
        raise ValueError("out must be float64")
    if not out.is_contiguous():
        raise ValueError("out must be contiguous")
    if out.numel() < 9:
        raise ValueError("out needs at least 9 elements")
    if out.device.index != torch.cuda.current_device():
        raise ValueError("out must be on the current CUDA device")


# ---- learned seed of the h iteration -----------------------------------------
def sph_mlp_set_weights(ctx, w):
    """Set the FP32 master parameters (MLP_NPARAM values); resets Adam."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(w, dtype=np.float32).ravel())
    _check(ctx, lib().sph_mlp_set_weights(ctx, a.ctypes.data_as(C.POINTER(C.c_float)), a.size))


def sph_mlp_get_weights(ctx):
    import numpy as np
    a = np.zeros(MLP_NPARAM, dtype=np.float32)
    _check(ctx, lib().sph_mlp_get_weights(ctx, a.ctypes.data_as(C.POINTER(C.c_float)), a.size))
    return a


def sph_mlp_set_seed_mode(ctx, mode):
    m = SEED_MODES[mode] if isinstance(mode, str) else int(mode)
    _check(ctx, lib().sph_mlp_set_seed_mode(ctx, m))


def sph_mlp_record(ctx, on=True, capacity=1 << 20, stride=1):
    _check(ctx, lib().sph_mlp_record(ctx, 1 if on else 0, int(capacity), int(stride)))


def sph_mlp_samples(ctx) -> int:
    n = C.c_int64()
    _check(ctx, lib().sph_mlp_samples(ctx, C.byref(n)))
    return n.value


def sph_mlp_get_samples(ctx, n=None):
    """Host copies (x (n, 4), y (n,)) of the first n samples held (all by default)."""
    import numpy as np
    if n is None:
        n = sph_mlp_samples(ctx)
    x = np.zeros((n, 4), dtype=np.float32)
    y = np.zeros(n, dtype=np.float32)
    _check(ctx, lib().sph_mlp_get_samples(ctx, x.ctypes.data_as(C.POINTER(C.c_float)),
                                          y.ctypes.data_as(C.POINTER(C.c_float)), int(n)))
    return x, y


def sph_mlp_load_samples(ctx, x, y, stream=None):
    """x: (n, 4) float32 device tensor, y: (n,) float32 device tensor."""
    x = x.contiguous()
    y = y.contiguous()
    _check(ctx, lib().sph_mlp_load_samples(ctx, C.c_void_p(x.data_ptr()),
                                           C.c_void_p(y.data_ptr()), int(y.numel()),
                                           _stream(stream)))


def sph_mlp_train(ctx, iters, batch=0, lr=1e-3, seed=0, stream=None):
    """Adam steps on the samples held; returns (first loss, last loss)."""
    l0 = C.c_double()
    l1 = C.c_double()
    _check(ctx, lib().sph_mlp_train(ctx, int(iters), int(batch), float(lr), int(seed),
                                    C.byref(l0), C.byref(l1), _stream(stream)))
    return l0.value, l1.value


def sph_mlp_grad(ctx, x, y, stream=None):
    """(gradient as numpy float32, loss) of the master network on device samples."""
    import numpy as np
    x = x.contiguous()
    y = y.contiguous()
    g = np.zeros(MLP_NPARAM, dtype=np.float32)
    loss = C.c_double()
    _check(ctx, lib().sph_mlp_grad(ctx, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                   int(y.numel()), g.ctypes.data_as(C.POINTER(C.c_float)),
                                   C.byref(loss), _stream(stream)))
    return g, loss.value


def sph_mlp_infer(ctx, x, out=None, stream=None):
    """Network outputs for the (n, 4) float32 device tensor x (tensor-core path)."""
    import torch
    x = x.contiguous()
    if out is None:
        out = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _check(ctx, lib().sph_mlp_infer(ctx, C.c_void_p(x.data_ptr()), int(x.shape[0]),
                                    C.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def sph_bucket_layout(ctx):
    """First particle of every bucket slot (plus the end sentinel), numpy int32."""
    import numpy as np
    ns = C.c_int64()
    lib().sph_bucket_layout(ctx, None, 0, C.byref(ns))
    first = np.zeros(ns.value + 1, dtype=np.int32)
    _check(ctx, lib().sph_bucket_layout(ctx, first.ctypes.data_as(C.POINTER(C.c_int32)),
                                        first.size, C.byref(ns)))
    return first


PHASES = ("keys", "sort", "permute", "layout", "buckets", "tree", "bob_refit", "walk",
          "density", "predict", "forces", "finalize", "kdk", "conserved")


def sph_set_profiling(ctx, on: bool):
    """Start (and clear) or stop per-phase device timing of plain calls."""
    _check(ctx, lib().sph_set_profiling(ctx, 1 if on else 0))


def sph_phase_times(ctx):
    """{phase: (total ms, launch groups)} accumulated while profiling."""
    st = c_stats()
    _check(ctx, lib().sph_get_stats(ctx, C.byref(st)))
    return {name: (st.phase_ms[k], int(st.phase_launches[k])) for k, name in enumerate(PHASES)}


def sph_step_rungs(ctx, parts: Particles, dt0: float, max_rung: int, stream=None):
    """One global step dt0 with hierarchical power-of-two substeps."""
    s = parts.c()
    _check(ctx, lib().sph_step_rungs(ctx, C.byref(s), float(dt0), int(max_rung),
                                     _stream(stream)))


def sph_set_fastgas(ctx, on: bool):
    """FastGas on (default) or off for the substeps of sph_step_rungs."""
    _check(ctx, lib().sph_set_fastgas(ctx, 1 if on else 0))


def sph_get_rungs(ctx, n: int):
    """Rungs of the first n particles (current order) as a numpy uint8 array."""
    import numpy as np
    a = np.zeros(int(n), dtype=np.uint8)
    _check(ctx, lib().sph_get_rungs(ctx, C.c_void_p(a.ctypes.data), int(n)))
    return a


def sph_set_list_arena(ctx, entries: int):
    """Capacity of the interaction-list overflow arena (entries of 4 bytes)."""
    _check(ctx, lib().sph_set_list_arena(ctx, int(entries)))


def sph_set_dt_old(ctx, dt_old: float):
    _check(ctx, lib().sph_set_dt_old(ctx, float(dt_old)))


def sph_get_stats(ctx) -> dict:
    st = c_stats()
    _check(ctx, lib().sph_get_stats(ctx, C.byref(st)))
    return {f: getattr(st, f) for f, _ in c_stats._fields_}


def sph_last_error(ctx) -> str:
    return lib().sph_last_error(ctx).decode()


class Simulation:
    """One problem on one GPU: owns the context and the particle tensors."""

    def __init__(self, prob, params: Params | None = None, device="cuda", capacity=None):
        self.params = params or Params.for_problem(prob)
        self.parts = Particles.from_problem(prob, device)
        self.ctx = sph_create(self.params, capacity or prob.n)
        self.t = 0.0

    def step(self, dt_fixed=0.0, stream=None) -> float:
        dt = sph_step(self.ctx, self.parts, dt_fixed, stream)
        self.t += dt
        return dt

    def stats(self):
        return sph_get_stats(self.ctx)

    def conserved(self, stream=None):
        return sph_reduce_conserved(self.ctx, self.parts, stream)

    def close(self):
        if self.ctx is not None:
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSimulation(Simulation):
    """Independent problems of uneven sizes stepped together: one launch per
    phase over all of them, optionally replayed from a captured CUDA graph."""

    def __init__(self, probs, params_list=None, device="cuda"):
        self.params_list = params_list or [Params.for_problem(q) for q in probs]
        self.parts, self.offsets = Particles.from_problems(probs, device)
        self.ninst = len(probs)
        self.ctx = sph_batch_create(self.params_list, self.offsets)
        self.t = [0.0] * self.ninst
        self.graph_stream = None

    def step(self, dt_fixed=0.0, stream=None) -> list:
        if self.graph_stream is not None:
            sph_graph_launch(self.ctx, self.graph_stream)
        else:
            sph_step(self.ctx, self.parts, dt_fixed, stream)
        dts = sph_batch_get_dt(self.ctx, self.ninst)
        self.t = [t + d for t, d in zip(self.t, dts)]
        return dts

    def capture(self, stream, dt_fixed=0.0):
        """Record one step as a CUDA graph on `stream` (not the default
        stream); later step() calls replay it there."""
        sph_graph_capture(self.ctx, self.parts, dt_fixed, stream)
        self.graph_stream = stream

    def conserved(self, stream=None):
        return sph_reduce_conserved(self.ctx, self.parts, stream, self.ninst)
