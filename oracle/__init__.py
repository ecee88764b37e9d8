"""FP64 brute-force SPH oracle -- TEST INFRASTRUCTURE, not product code.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg
of ``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_2511_11425_gb300``; it imports nothing from it.

What it computes, and where the paper defines it (arXiv:2511.11425):

* kernels W(r,h) = w(r/h)/h^3 with compact support h (Sec. 2.3: cubic spline,
  Wendland C2/C4/C6; the paper prints no formulas, the textbook 3D forms are
  used)                                                -> ``kernel_eval``
* rho_i = sum_j m_j W_ij(h_i) with h_i from Newton-Raphson on the constant
  kernel mass 4/3 pi h^3 rho = N_ngb m, grad-h term Omega (Sec. 2.3.3)
                                                       -> ``density_h``
* P = (gamma-1) rho u (Sec. 2.3.1)                     -> ``eos``
* momentum / PdV / artificial-viscosity equations and the time-step criteria
  (Sec. 2.3.5, Sec. 2.3.6, Eq. courant_condition)      -> ``forces``
* kick-drift-kick with the embedded predictor (Sec. 2.3.6, single global
  time step)                                           -> ``Simulation.step``
* conserved totals                                     -> ``conserved``
* interface correction: kernel imbalance, exp(-I^2)-weighted kernel averages
  of T and P, corrected density from the EOS (Sec. 2.3.4)
                                                       -> ``interface_correction``

The heavy loops are in ``sph_oracle.c`` (plain C, OpenMP over sinks); this
file only marshals numpy arrays.  Exact Riemann and Sedov-Taylor solutions
live in ``oracle.riemann`` and ``oracle.sedov``.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math

import numpy as np

from . import build as _build

KERNELS = {"wc2": 0, "wc4": 1, "wc6": 2, "m4": 3}


class _Params(C.Structure):
    _fields_ = [
        ("kernel", C.c_int), ("max_iter", C.c_int),
        ("n_ngb", C.c_double), ("gamma", C.c_double),
        ("alpha", C.c_double), ("beta", C.c_double), ("eps_av", C.c_double),
        ("eta_courant", C.c_double), ("eta_acc", C.c_double),
        ("h_rel_tol", C.c_double),
        ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
        ("periodic", C.c_int * 3), ("pad_", C.c_int),
    ]


@dataclasses.dataclass
class Params:
    """Physical and numerical parameters of one problem (oracle side)."""
    kernel: str = "wc2"
    n_ngb: float = 64.0
    gamma: float = 5.0 / 3.0
    alpha: float = 1.0
    beta: float = 2.0
    eps_av: float = 0.01
    eta_courant: float = 0.15
    eta_acc: float = 0.2
    h_rel_tol: float = 1e-12
    max_iter: int = 200
    box_lo: tuple = (0.0, 0.0, 0.0)
    box_hi: tuple = (1.0, 1.0, 1.0)
    periodic: tuple = (1, 1, 1)

    def c(self) -> _Params:
        p = _Params()
        p.kernel = KERNELS[self.kernel]
        p.max_iter = int(self.max_iter)
        for f in ("n_ngb", "gamma", "alpha", "beta", "eps_av", "eta_courant",
                  "eta_acc", "h_rel_tol"):
            setattr(p, f, float(getattr(self, f)))
        for a in range(3):
            p.box_lo[a] = float(self.box_lo[a])
            p.box_hi[a] = float(self.box_hi[a])
            p.periodic[a] = int(bool(self.periodic[a]))
        return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int64)
        i32p = C.POINTER(C.c_int32)
        pp = C.POINTER(_Params)
        L.orc_kernel_eval.argtypes = [C.c_int, C.c_int64, dp, dp, dp]
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = C.c_int
        L.orc_density_h.argtypes = [pp, C.c_int64, dp, dp, C.c_int64, ip, dp,
                                    dp, dp, dp, ip, i32p]
        L.orc_density_h.restype = C.c_int64
        L.orc_density_at.argtypes = [pp, C.c_int64, dp, dp, C.c_int64, ip, dp, dp, dp, ip]
        L.orc_neighbours.argtypes = [pp, C.c_int64, dp, C.c_int64, C.c_double, C.c_int64,
                                     ip, dp]
        L.orc_neighbours.restype = C.c_int64
        L.orc_forces.argtypes = [pp, C.c_int64, dp, dp, dp, dp, dp, dp, dp, C.c_int64, ip,
                                 dp, dp, dp, dp, dp, dp]
        L.orc_imbalance.argtypes = [pp, C.c_int64, dp, dp, dp, i32p, C.c_double, C.c_int64,
                                    ip, dp]
        L.orc_interface_averages.argtypes = [pp, C.c_int64, dp, dp, dp, dp, dp, C.c_int64, ip,
                                             dp, dp]
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def _sinks(n, sinks):
    if sinks is None:
        return None, n
    s = np.ascontiguousarray(sinks, dtype=np.int64)
    return s, len(s)


def kernel_eval(kernel: str, q):
    """Dimensionless w(q) and w'(q) of the named kernel (support q < 1)."""
    q = _d(q).ravel()
    w = np.empty_like(q)
    dw = np.empty_like(q)
    lib().orc_kernel_eval(KERNELS[kernel], len(q), _ptr(q), _ptr(w), _ptr(dw))
    return w, dw


def density_h(params: Params, pos, m, h_seed, sinks=None):
    """Newton-Raphson smoothing length + density for the sinks (all if None).

    Returns dict(h, rho, omega, nngb, iters, failed); arrays follow ``sinks``.
    """
    pos = _d(pos).reshape(-1, 3)
    m = _d(m)
    n = len(m)
    s, ns = _sinks(n, sinks)
    hs = _d(h_seed) if np.ndim(h_seed) else np.full(ns, float(h_seed))
    if hs.shape[0] != ns:
        hs = _d(hs[s]) if s is not None else hs
    out = {k: np.empty(ns) for k in ("h", "rho", "omega")}
    nngb = np.empty(ns, dtype=np.int64)
    iters = np.empty(ns, dtype=np.int32)
    cp = params.c()
    failed = lib().orc_density_h(C.byref(cp), n, _ptr(pos), _ptr(m), ns,
                                 _ptr(s, C.c_int64) if s is not None else None, _ptr(hs),
                                 _ptr(out["h"]), _ptr(out["rho"]), _ptr(out["omega"]),
                                 _ptr(nngb, C.c_int64), _ptr(iters, C.c_int32))
    out.update(nngb=nngb, iters=iters, failed=int(failed))
    return out


def density_at(params: Params, pos, m, h, sinks=None):
    """rho, Omega and neighbour count at the given h (no iteration)."""
    pos = _d(pos).reshape(-1, 3)
    m = _d(m)
    n = len(m)
    s, ns = _sinks(n, sinks)
    h = _d(h)
    if h.shape[0] != ns:
        h = _d(h[s])
    rho = np.empty(ns)
    om = np.empty(ns)
    nngb = np.empty(ns, dtype=np.int64)
    cp = params.c()
    lib().orc_density_at(C.byref(cp), n, _ptr(pos), _ptr(m), ns,
                         _ptr(s, C.c_int64) if s is not None else None, _ptr(h),
                         _ptr(rho), _ptr(om), _ptr(nngb, C.c_int64))
    return {"rho": rho, "omega": om, "nngb": nngb}


def neighbours(params: Params, pos, i: int, h: float, cap: int = 4096):
    """Sorted indices j != i with r_ij < h, and min_j |r_ij - h|/h."""
    pos = _d(pos).reshape(-1, 3)
    out = np.empty(cap, dtype=np.int64)
    mg = C.c_double()
    cp = params.c()
    c = lib().orc_neighbours(C.byref(cp), len(pos), _ptr(pos), int(i), float(h), cap,
                             _ptr(out, C.c_int64), C.byref(mg))
    if c > cap:
        return neighbours(params, pos, i, h, cap=int(c) + 16)
    return out[:c].copy(), mg.value


def eos(gamma, rho, u):
    """Ideal gas (Sec. 2.3.1): P = (gamma-1) rho u, c = sqrt(gamma P / rho)."""
    P = (gamma - 1.0) * np.asarray(rho) * np.asarray(u)
    return P, np.sqrt(gamma * P / np.asarray(rho))


def forces(params: Params, pos, vel, m, h, rho, omega, u, sinks=None):
    """Accelerations, du/dt (hydro, viscous), div v and dt_i for the sinks.

    ``vel`` and ``u`` are the predicted values; every array covers ALL
    particles (sources); results follow ``sinks``.
    """
    pos = _d(pos).reshape(-1, 3)
    vel = _d(vel).reshape(-1, 3)
    m, h, rho, omega, u = (_d(a) for a in (m, h, rho, omega, u))
    n = len(m)
    s, ns = _sinks(n, sinks)
    acc = np.empty((ns, 3))
    out = {k: np.empty(ns) for k in ("dudt_h", "dudt_av", "divv", "dt", "vdw_abs")}
    cp = params.c()
    lib().orc_forces(C.byref(cp), n, _ptr(pos), _ptr(vel), _ptr(m), _ptr(h), _ptr(rho),
                     _ptr(omega), _ptr(u), ns,
                     _ptr(s, C.c_int64) if s is not None else None,
                     _ptr(acc), _ptr(out["dudt_h"]), _ptr(out["dudt_av"]),
                     _ptr(out["divv"]), _ptr(out["dt"]), _ptr(out["vdw_abs"]))
    out["a"] = acc
    # conditioning of the PdV / div v sums (sum of the terms' magnitudes),
    # in the units of dudt_h and divv
    si = s if s is not None else np.arange(n)
    P = (params.gamma - 1.0) * rho[si] * u[si]
    out["dudt_h_scale"] = np.abs(P / (omega[si] * rho[si] ** 2)) * out["vdw_abs"]
    out["divv_scale"] = out["vdw_abs"] / np.abs(omega[si] * rho[si])
    return out


def imbalance_norm(kernel: str) -> float:
    """alpha of Eq. Kernel_imbalance for `kernel`: the reciprocal of the raw
    imbalance of a particle on a flat interface between two uniform
    half-spaces of different material, 2 pi int_0^1 w(q) q^3 dq (the
    numerator is 2 rho int_{z>0} z W dV = 2 rho pi h int w q^3 dq, the
    denominator h rho), so that such a particle has I = 1.  Gauss-Legendre
    quadrature of the kernel as the oracle evaluates it, on [0, 1/2] and
    [1/2, 1] separately (exact for the piecewise cubic spline as well)."""
    x, wq = np.polynomial.legendre.leggauss(32)
    total = 0.0
    for a, b in ((0.0, 0.5), (0.5, 1.0)):
        q = a + 0.5 * (b - a) * (x + 1.0)
        w, _ = kernel_eval(kernel, q)
        total += 0.5 * (b - a) * float(np.sum(wq * w * q ** 3))
    return 1.0 / (2.0 * math.pi * total)


def imbalance(params: Params, pos, m, h, mat, alpha=None, sinks=None):
    """Kernel imbalance I_i (Sec. 2.3.4, Eq. Kernel_imbalance)."""
    pos = _d(pos).reshape(-1, 3)
    m, h = _d(m), _d(h)
    mat = np.ascontiguousarray(mat, dtype=np.int32)
    n = len(m)
    s, ns = _sinks(n, sinks)
    a = imbalance_norm(params.kernel) if alpha is None else float(alpha)
    out = np.empty(ns)
    cp = params.c()
    lib().orc_imbalance(C.byref(cp), n, _ptr(pos), _ptr(m), _ptr(h),
                        mat.ctypes.data_as(C.POINTER(C.c_int32)), a, ns,
                        _ptr(s, C.c_int64) if s is not None else None, _ptr(out))
    return out


def interface_correction(params: Params, pos, m, h, rho, u, mat, r_gas, alpha=None):
    """Interface correction of Sec. 2.3.4 for every particle, ideal gases
    with one gamma and a gas constant per material (T = (gamma-1) u / R):
    I from Eq. Kernel_imbalance, Tbar and Pbar kernel averages weighted by
    exp(-I^2), P~ = e^{-I^2} P + (1 - e^{-I^2}) Pbar (T~ likewise), and the
    corrected density from the EOS, rho~ = P~ / (R T~)."""
    pos = _d(pos).reshape(-1, 3)
    m, h, rho, u = _d(m), _d(h), _d(rho), _d(u)
    mat = np.ascontiguousarray(mat, dtype=np.int32)
    R = np.asarray(r_gas, dtype=np.float64)[mat]
    g = params.gamma
    P = (g - 1.0) * rho * u
    T = (g - 1.0) * u / R
    I = imbalance(params, pos, m, h, mat, alpha)
    eI = np.exp(-I * I)
    n = len(m)
    tbar = np.empty(n)
    pbar = np.empty(n)
    cp = params.c()
    lib().orc_interface_averages(C.byref(cp), n, _ptr(pos), _ptr(h), _ptr(eI), _ptr(T), _ptr(P),
                                 n, None, _ptr(tbar), _ptr(pbar))
    Pt = eI * P + (1.0 - eI) * pbar
    Tt = eI * T + (1.0 - eI) * tbar
    return {"I": I, "eI": eI, "P": P, "T": T, "Tbar": tbar, "Pbar": pbar, "P_corr": Pt,
            "T_corr": Tt, "rho_corr": Pt / (R * Tt)}


def conserved(pos, vel, m, u):
    """Totals [M, Px, Py, Pz, Lx, Ly, Lz, E_kin, E_int] in FP64."""
    pos = _d(pos).reshape(-1, 3)
    vel = _d(vel).reshape(-1, 3)
    m = _d(m)
    u = _d(u)
    mom = (m[:, None] * vel).sum(0)
    L = (m[:, None] * np.cross(pos, vel)).sum(0)
    ek = 0.5 * (m * (vel * vel).sum(1)).sum()
    ei = (m * u).sum()
    return np.array([m.sum(), *mom, *L, ek, ei])


class Simulation:
    """Global-time-step kick-drift-kick with the embedded predictor (Sec. 2.3.6).

    State between steps: x_i, v_{i-1/2}, u_{i-1/2}, the last derivatives
    a_{i-1}, udot_{i-1} and the last step size.  One ``step``:
      1 density pass at x_i                               (h, rho, Omega)
      2 predict v, u to time i with the old derivatives and half the old step
      3 forces with the predicted v, u                    (a_i, udot_i, dt_i)
      4 closing kick over half the old step
      5 new step = dt_fixed, else min_i dt_i
      6 opening kick over half the new step
      7 drift x over the new step (periodic wrap)
    At t=0 the old step is zero, so v_pred = v_0 and the closing kick vanishes.
    energy='pdv' kicks u with du/dt|H + du/dt|Pi; energy='isentropic' first
    moves u along its adiabat to the new density, u <- u (rho/rho_old)^(gamma-1),
    then kicks with du/dt|Pi only (Sec. 2.3.5, entropy-conserving update).

    density='evolved' is the variant of Sec. 2.3.3 in which the density is
    integrated with the mass conservation equation drho/dt = -rho div v
    instead of taken from the kernel sum; the density pass still gives h and
    Omega.  rho is then state like u: the first step starts it from the
    kernel sum, the predictor moves it by half the old step with the rate
    -rho div v_old (div v of the last force evaluation), the forces use that
    predicted rho, and the two half kicks use the new rate -rho_pred div v.
    """

    def __init__(self, params: Params, pos, vel, m, u, h0, energy="pdv", density="summed"):
        self.p = params
        self.x = _d(pos).reshape(-1, 3).copy()
        self.v = _d(vel).reshape(-1, 3).copy()
        self.m = _d(m).copy()
        self.u = _d(u).copy()
        self.h = _d(h0).copy() if np.ndim(h0) else np.full(len(self.m), float(h0))
        n = len(self.m)
        self.a = np.zeros((n, 3))
        self.udot = np.zeros(n)
        self.rho_old = None
        self.dt_old = 0.0
        self.t = 0.0
        self.energy = energy
        if density not in ("summed", "evolved"):
            raise ValueError("density must be 'summed' or 'evolved'")
        if density == "evolved" and energy != "pdv":
            raise ValueError("the evolved density is integrated with the PdV energy equation")
        self.density = density
        self.rho = None      # evolved density (state between steps)
        self.divv_old = None  # div v of the last force evaluation
        self.last = None

    def step(self, dt_fixed=None):
        p = self.p
        d = density_h(p, self.x, self.m, self.h)
        if d["failed"]:
            raise RuntimeError("oracle Newton iteration did not converge")
        self.h = d["h"]
        if self.energy == "isentropic" and self.rho_old is not None:
            self.u = self.u * (d["rho"] / self.rho_old) ** (p.gamma - 1.0)
        v_pred = self.v + 0.5 * self.dt_old * self.a
        u_pred = self.u + 0.5 * self.dt_old * self.udot
        if self.density == "evolved":
            if self.rho is None:
                self.rho = d["rho"].copy()
                self.divv_old = np.zeros(len(self.m))
            rho_f = self.rho * (1.0 - 0.5 * self.dt_old * self.divv_old)
        else:
            rho_f = d["rho"]
        f = forces(p, self.x, v_pred, self.m, d["h"], rho_f, d["omega"], u_pred)
        udot = f["dudt_av"] if self.energy == "isentropic" else f["dudt_h"] + f["dudt_av"]
        self.v = self.v + 0.5 * self.dt_old * f["a"]
        self.u = self.u + 0.5 * self.dt_old * udot
        dt = float(dt_fixed) if dt_fixed else float(f["dt"].min())
        self.v = self.v + 0.5 * dt * f["a"]
        self.u = self.u + 0.5 * dt * udot
        if self.density == "evolved":
            rhodot = -rho_f * f["divv"]          # mass conservation equation
            self.rho = self.rho + 0.5 * (self.dt_old + dt) * rhodot
            self.divv_old = f["divv"]
        self.x = self.x + dt * self.v
        for a in range(3):
            if p.periodic[a]:
                lo, hi = p.box_lo[a], p.box_hi[a]
                self.x[:, a] = lo + np.mod(self.x[:, a] - lo, hi - lo)
        self.a = f["a"]
        self.udot = udot
        self.rho_old = d["rho"]
        self.dt_old = dt
        self.t += dt
        self.last = {**d, **f, "v_pred": v_pred, "u_pred": u_pred, "rho_forces": rho_f}
        return dt


def sod_h_estimate(m, rho, n_ngb):
    """h from the constant-mass criterion for a known density (used by tests)."""
    return (3.0 * n_ngb * np.asarray(m) / (4.0 * math.pi * np.asarray(rho))) ** (1.0 / 3.0)


def force_partners_max(params: Params, pos, h, values):
    """max over the force partners j of each particle (r_ij < max(h_i, h_j),
    j != i, minimum image) of values[j]; -1 where there is none.  Brute
    force in numpy (test sizes)."""
    pos = _d(pos).reshape(-1, 3)
    h = _d(h)
    n = len(h)
    L = np.array(params.box_hi, dtype=np.float64) - np.array(params.box_lo, dtype=np.float64)
    per = np.array(params.periodic, dtype=bool)
    out = np.full(n, -1, dtype=np.int64)
    vals = np.asarray(values, dtype=np.int64)
    for i in range(n):
        d = pos - pos[i]
        d[:, per] -= L[per] * np.round(d[:, per] / L[per])
        r = np.sqrt((d * d).sum(1))
        nb = (r < np.maximum(h[i], h)) & (np.arange(n) != i)
        if np.any(nb):
            out[i] = int(vals[nb].max())
    return out


class RungSimulation:
    """Hierarchical kick-drift-kick with power-of-two steps (Sec. 2.3.6).

    A global step dt0 is cut into 2^R substeps of delta = dt0 / 2^R; a
    particle on rung r has the step 2^(R-r) delta and is active at the
    substeps s with s mod 2^(R-r) = 0.  Every substep:
      1 density pass for all particles
      2 predictor for all: the time tau since the particle's last boundary
        (its whole period when it is active now), v_pred = v + (tau - T/2) a,
        u_pred likewise, T = 2^(R-r) delta the period of its current rung
        (v, u are half-step values; at the start of the run v_pred = v)
      3 forces for all; the active particles take the new derivatives,
        the others keep theirs
      4 active particles: closing kick over T/2 (none at the start), new
        rung r_des = ceil(log2(dt0 / dt_i)) clamped to [0, R], raised to at
        least (max rung of its force partners) - 2 (Saitoh & Makino's
        limiter as the paper applies it); a lower rung only to a rung whose
        period divides s (the lowest such rung >= r_des), then the opening
        kick over half the new period
      5 drift of every particle over delta.
    """

    def __init__(self, params: Params, pos, vel, m, u, h0, max_rung):
        self.p = params
        self.x = _d(pos).reshape(-1, 3).copy()
        self.v = _d(vel).reshape(-1, 3).copy()
        self.m = _d(m).copy()
        self.u = _d(u).copy()
        n = len(self.m)
        self.h = _d(h0).copy() if np.ndim(h0) else np.full(n, float(h0))
        self.a = np.zeros((n, 3))
        self.udot = np.zeros(n)
        self.R = int(max_rung)
        self.rung = np.zeros(n, dtype=np.int64)
        self.started = False
        self.t = 0.0
        self.log = []   # per substep: (active indices, their new rungs, log2(dt0 / dt_i))

    def global_step(self, dt0):
        p = self.p
        R = self.R
        delta = dt0 / 2 ** R
        for s in range(2 ** R):
            d = density_h(p, self.x, self.m, self.h)
            if d["failed"]:
                raise RuntimeError("oracle Newton iteration did not converge")
            self.h = d["h"]
            per = 2 ** (R - self.rung)
            phi = s % per
            active = phi == 0
            if self.started:
                tau = np.where(active, per, phi) * delta
                off = tau - 0.5 * per * delta
                v_pred = self.v + off[:, None] * self.a
                u_pred = self.u + off * self.udot
            else:
                v_pred = self.v.copy()
                u_pred = self.u.copy()
            f = forces(p, self.x, v_pred, self.m, d["h"], d["rho"], d["omega"], u_pred)
            udot = f["dudt_h"] + f["dudt_av"]
            partner = force_partners_max(p, self.x, d["h"], self.rung)
            act = np.nonzero(active)[0]
            self.a[act] = f["a"][act]
            self.udot[act] = udot[act]
            if self.started:
                half = 0.5 * per[act] * delta
                self.v[act] += half[:, None] * self.a[act]
                self.u[act] += half * self.udot[act]
            ratio = np.log2(dt0 / f["dt"][act])
            want = np.clip(np.ceil(ratio), 0, R).astype(np.int64)
            want = np.maximum(want, partner[act] - 2)
            want = np.minimum(want, R)
            new = self.rung[act].copy()
            for k, i in enumerate(act):
                r_old, r_des = self.rung[i], want[k]
                if r_des >= r_old:
                    new[k] = r_des
                else:
                    for r in range(r_des, r_old + 1):
                        if s % 2 ** (R - r) == 0:
                            new[k] = r
                            break
            self.rung[act] = new
            half = 0.5 * 2 ** (R - new) * delta
            self.v[act] += half[:, None] * self.a[act]
            self.u[act] += half * self.udot[act]
            self.x = self.x + delta * self.v
            for ax in range(3):
                if p.periodic[ax]:
                    lo, hi = p.box_lo[ax], p.box_hi[ax]
                    self.x[:, ax] = lo + np.mod(self.x[:, ax] - lo, hi - lo)
            self.started = True
            self.t += delta
            self.log.append((act, new.copy(), ratio))
        return 2 ** R
