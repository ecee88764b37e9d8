"""Seeded synthetic initial conditions shaped like the paper's test problems.

This module is shared by the tests, the benchmark and the oracle checks.  It
holds no SPH arithmetic: it only lays particles on lattices, jitters them
with a counter-based generator, and assigns masses, velocities and internal
energies from the problem statement.  The smoothing-length seed it returns is
a plain multiple of the local lattice spacing; the density pass converges
from it.

Problems (sizes as used by the tests and the benchmark):
  sod       3D Sod tube, gamma 1.4, left rho=P=1 (dx = 1/192, 96x12x12),
            right rho=0.125, P=0.1 (2 dx, 48x6x6), equal masses, 15,552
            particles, periodic on all axes (Sec. 3.2)
  sedov     periodic unit box, n^3 lattice, rho=1, u=1e-6 plus E=1 deposited
            with a smooth compact bump of radius 2 spacings round the centre,
            gamma 5/3 (Sec. 3.3)
  kh        n^3 periodic unit box, band 0.25<y<0.75 twice as dense (double
            mass, same spacing), opposing x velocities +-0.5, P=2.5,
            v_y = 0.01 sin(4 pi x), gamma 5/3 (Sec. 3.8 geometry)
  uniform   jittered periodic lattice with small random velocities
  collision two spheres with rho ~ 1/r truncated at r=0.02, radii 1 and 0.5,
            approaching at Mach 3, impact parameter 0.5, open boundaries
  batch     list of independent sod / sedov instances with log-uniform sizes
  soundwave linear travelling sound wave, N BCC (or cubic) cells along x and
            16 across, A = 1e-3, gamma 5/3, Wendland C6 with 400 neighbours
            (Sec. 3.1)

Random numbers: SplitMix64 (Steele, Lea & Flood 2014) on the counter
seed*2^32 + 4*index + stream, mapped to [0,1) with the top 53 bits.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each uint64 counter value."""
    with np.errstate(over="ignore"):
        z = (np.asarray(counter, dtype=np.uint64) + _GOLDEN).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, index: np.ndarray, stream: int) -> np.ndarray:
    """Uniform [0,1) doubles keyed on (seed, index, stream)."""
    with np.errstate(over="ignore"):
        c = (np.uint64(seed) << np.uint64(32)) + np.asarray(index, dtype=np.uint64) * np.uint64(4) \
            + np.uint64(stream)
    return (splitmix64(c) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class Problem:
    """Particles plus the problem's parameters (all arrays in input order)."""
    name: str
    pos: np.ndarray          # (N,3) float64
    vel: np.ndarray          # (N,3) float64
    u: np.ndarray            # (N,)  float64 specific internal energy
    m: np.ndarray            # (N,)  float64 masses
    h0: np.ndarray           # (N,)  float64 smoothing-length seed
    box_lo: tuple
    box_hi: tuple
    periodic: tuple
    gamma: float
    alpha: float
    beta: float
    kernel: str = "wc2"
    n_ngb: float = 64.0
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.m)


def _lattice(nx, ny, nz, lo, spacing):
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    pts = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64) + 0.5
    return np.asarray(lo, dtype=np.float64) + pts * spacing


def _jitter(pos, spacing, seed, first_index, amp=1e-3):
    n = len(pos)
    idx = np.arange(first_index, first_index + n, dtype=np.uint64)
    out = pos.copy()
    sp = np.broadcast_to(np.asarray(spacing, dtype=np.float64), (n,))
    for a in range(3):
        out[:, a] += (2.0 * uniform01(seed, idx, a) - 1.0) * amp * sp
    return out


def _wrap(pos, lo, hi, periodic):
    for a in range(3):
        if periodic[a]:
            pos[:, a] = lo[a] + np.mod(pos[:, a] - lo[a], hi[a] - lo[a])
    return pos


def sod(seed: int = 2511, nl: int = 12, length_cells: int = 96, gamma: float = 1.4,
        alpha: float = 1.5, beta: float = 3.0, jitter: float = 1e-3, dx: float = None) -> Problem:
    """Sod tube: left block length_cells x nl x nl at dx, right block at 2 dx.

    Defaults give dx = 1/192 (each half 1/2 long), a 1/16 cross-section and
    N = 15,552.  With dx given, each half is length_cells * dx long.
    """
    if nl % 2 or length_cells % 2:
        raise ValueError("nl and length_cells must be even")
    if dx is None:
        dx = 0.5 / length_cells
    half = length_cells * dx
    L_yz = nl * dx
    left = _lattice(length_cells, nl, nl, (-half, 0.0, 0.0), dx)
    right = _lattice(length_cells // 2, nl // 2, nl // 2, (0.0, 0.0, 0.0), 2 * dx)
    pos = np.concatenate([left, right])
    sp = np.concatenate([np.full(len(left), dx), np.full(len(right), 2 * dx)])
    pos = _jitter(pos, sp, seed, 0, jitter)
    lo, hi, per = (-half, 0.0, 0.0), (half, L_yz, L_yz), (1, 1, 1)
    pos = _wrap(pos, lo, hi, per)
    n = len(pos)
    m = np.full(n, dx ** 3)
    rho = np.where(np.arange(n) < len(left), 1.0, 0.125)
    P = np.where(np.arange(n) < len(left), 1.0, 0.1)
    u = P / ((gamma - 1.0) * rho)
    return Problem("sod", pos, np.zeros((n, 3)), u, m, 2.5 * sp, lo, hi, per,
                   gamma, alpha, beta, extra={"dx": dx, "n_left": len(left)})


def sedov(n: int = 64, seed: int = 2511, E: float = 1.0, gamma: float = 5.0 / 3.0,
          alpha: float = 1.0, beta: float = 2.0, u0: float = 1e-6,
          jitter: float = 1e-3) -> Problem:
    """Sedov-Taylor blast in the periodic unit box on an n^3 lattice."""
    dx = 1.0 / n
    pos = _jitter(_lattice(n, n, n, (0.0, 0.0, 0.0), dx), dx, seed, 0, jitter)
    lo, hi, per = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (1, 1, 1)
    pos = _wrap(pos, lo, hi, per)
    N = len(pos)
    m = np.full(N, 1.0 / N)
    r = np.linalg.norm(pos - 0.5, axis=1)
    R = 2.0 * dx
    wgt = np.where(r < R, (1.0 - (r / R) ** 2) ** 2, 0.0)
    u = u0 + E * wgt / (m * wgt.sum())
    return Problem("sedov", pos, np.zeros((N, 3)), u, m, np.full(N, 2.5 * dx), lo, hi, per,
                   gamma, alpha, beta, extra={"dx": dx, "E": E})


def kh(n: int = 128, seed: int = 2511, gamma: float = 5.0 / 3.0, alpha: float = 1.0,
       beta: float = 2.0, P0: float = 2.5, jitter: float = 1e-3) -> Problem:
    """Kelvin-Helmholtz shear layer in the periodic unit box (n^3 particles)."""
    dx = 1.0 / n
    pos = _jitter(_lattice(n, n, n, (0.0, 0.0, 0.0), dx), dx, seed, 0, jitter)
    lo, hi, per = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (1, 1, 1)
    pos = _wrap(pos, lo, hi, per)
    N = len(pos)
    band = (pos[:, 1] > 0.25) & (pos[:, 1] < 0.75)
    rho = np.where(band, 2.0, 1.0)
    m = rho * dx ** 3
    vel = np.zeros((N, 3))
    vel[:, 0] = np.where(band, 0.5, -0.5)
    vel[:, 1] = 0.01 * np.sin(4.0 * math.pi * pos[:, 0])
    u = P0 / ((gamma - 1.0) * rho)
    return Problem("kh", pos, vel, u, m, np.full(N, 2.5 * dx), lo, hi, per, gamma, alpha, beta,
                   extra={"dx": dx})


def soundwave(N: int = 32, lattice: str = "bcc", A: float = 1e-3, ncross: int = 16,
              gamma: float = 5.0 / 3.0, kernel: str = "wc6", n_ngb: float = 400.0,
              alpha: float = 1.0, beta: float = 2.0) -> Problem:
    """Linear travelling sound wave (Sec. 3.1): periodic box of unit length in
    x and ncross cells of side 1/N in y and z, N cells in x (BCC: two
    particles per cell, or a primitive cubic lattice), unit density and sound
    speed (P0 = 1/gamma), equal masses.  Particles are displaced by
    dx = -(A / 2 pi) cos(2 pi x - pi/2), which gives rho = 1 + A cos(2 pi x)
    to first order; P = P0 (1 + gamma A cos(2 pi x)) fixes u, and the wave
    travels in +x with v_x = A cos(2 pi x) (the sound speed times the
    relative density amplitude)."""
    if lattice not in ("bcc", "cubic"):
        raise ValueError("lattice must be 'bcc' or 'cubic'")
    d = 1.0 / N
    base = _lattice(N, ncross, ncross, (0.0, 0.0, 0.0), d)
    if lattice == "bcc":
        pos = np.concatenate([base - 0.25 * d, base + 0.25 * d])
    else:
        pos = base
    x0 = pos[:, 0].copy()
    pos[:, 0] = x0 - A / (2.0 * math.pi) * np.cos(2.0 * math.pi * x0 - 0.5 * math.pi)
    lo, hi, per = (0.0, 0.0, 0.0), (1.0, ncross * d, ncross * d), (1, 1, 1)
    pos = _wrap(pos, lo, hi, per)
    n = len(pos)
    vol = 1.0 * (ncross * d) ** 2
    m = np.full(n, vol / n)
    xc = pos[:, 0]
    rho = 1.0 + A * np.cos(2.0 * math.pi * xc)
    P0 = 1.0 / gamma
    P = P0 * (1.0 + gamma * A * np.cos(2.0 * math.pi * xc))
    u = P / ((gamma - 1.0) * rho)
    vel = np.zeros((n, 3))
    vel[:, 0] = A * np.cos(2.0 * math.pi * xc)
    spacing = (vol / n) ** (1.0 / 3.0)
    h0 = np.full(n, (3.0 * n_ngb / (4.0 * math.pi)) ** (1.0 / 3.0) * spacing)
    return Problem("soundwave", pos, vel, u, m, h0, lo, hi, per, gamma, alpha, beta,
                   kernel=kernel, n_ngb=n_ngb, extra={"N": N, "A": A, "lattice": lattice})


def uniform(n: int = 16, seed: int = 7, L: float = 1.0, vamp: float = 0.1, u0: float = 1.0,
            gamma: float = 5.0 / 3.0, alpha: float = 1.0, beta: float = 2.0,
            jitter: float = 0.2, periodic=(1, 1, 1)) -> Problem:
    """Jittered periodic lattice with random velocities and energies (test helper)."""
    dx = L / n
    pos = _jitter(_lattice(n, n, n, (0.0, 0.0, 0.0), dx), dx, seed, 0, jitter)
    lo, hi = (0.0, 0.0, 0.0), (L, L, L)
    pos = _wrap(pos, lo, hi, periodic)
    N = len(pos)
    idx = np.arange(N, dtype=np.uint64)
    vel = np.stack([vamp * (2.0 * uniform01(seed + 1, idx, a) - 1.0) for a in range(3)], 1)
    u = u0 * (0.5 + uniform01(seed + 2, idx, 0))
    m = (1.0 + 0.5 * uniform01(seed + 3, idx, 0)) * dx ** 3
    return Problem("uniform", pos, vel, u, m, np.full(N, 2.5 * dx), lo, hi, tuple(periodic),
                   gamma, alpha, beta, extra={"dx": dx})


def _sphere_radii(N, R, r_core, seed, stream):
    """Radii with density ~ 1/r on r_core < r < R (enclosed mass ~ r^2)."""
    x = uniform01(seed, np.arange(N, dtype=np.uint64), stream)
    return np.sqrt(r_core ** 2 + x * (R ** 2 - r_core ** 2))


def _sphere(N, R, seed, stream0):
    r = _sphere_radii(N, R, 0.02 * R, seed, stream0)
    idx = np.arange(N, dtype=np.uint64)
    cz = 2.0 * uniform01(seed, idx, stream0 + 1) - 1.0
    ph = 2.0 * math.pi * uniform01(seed, idx, stream0 + 2)
    s = np.sqrt(1.0 - cz * cz)
    return np.stack([r * s * np.cos(ph), r * s * np.sin(ph), r * cz], 1), r


def collision(n_total: int = 8_000_000, seed: int = 2511, gamma: float = 5.0 / 3.0,
              alpha: float = 1.0, beta: float = 2.0, u0: float = 0.05) -> Problem:
    """Two 1/r spheres (radii 1 and 0.5, masses 1 and 0.25, equal particle mass).

    The small sphere moves at 3 sound speeds of u0 towards the large one with
    impact parameter 0.5; positions are random (inverse-CDF radii, isotropic
    directions), so the first density pass relaxes them.
    """
    n1 = int(round(n_total * 0.8))
    n2 = n_total - n1
    p1, r1 = _sphere(n1, 1.0, seed, 0)
    p2, r2 = _sphere(n2, 0.5, seed + 1, 0)
    c_s = math.sqrt(gamma * (gamma - 1.0) * u0)
    v_rel = 3.0 * c_s
    p2 = p2 + np.array([1.6, 0.5, 0.0])
    pos = np.concatenate([p1, p2])
    N = len(pos)
    vel = np.zeros((N, 3))
    vel[n1:, 0] = -v_rel
    m = np.full(N, 1.25 / N)
    r = np.concatenate([r1, r2 / 0.5])
    rho_ic = 1.0 / (2.0 * math.pi * np.maximum(r, 0.02))
    spacing = (m / rho_ic) ** (1.0 / 3.0)
    lo = tuple(pos.min(0) - 1e-6)
    hi = tuple(pos.max(0) + 1e-6)
    return Problem("collision", pos, vel, np.full(N, u0), m, 2.5 * spacing, lo, hi, (0, 0, 0),
                   gamma, alpha, beta, extra={"n1": n1, "v_rel": v_rel})


def batch(n_inst: int = 256, lo_n: int = 2000, hi_n: int = 200000, seed: int = 2511):
    """Independent sod / sedov instances with log-uniform particle counts.

    Even instances are Sod tubes with the 12/6 cross-section and dx = 1/192
    whose length grows with the count (162 particles per left-lattice
    column); odd instances are Sedov blasts on round(N^(1/3))^3 lattices."""
    idx = np.arange(n_inst, dtype=np.uint64)
    x = uniform01(seed, idx, 3)
    target = np.exp(math.log(lo_n) + x * (math.log(hi_n) - math.log(lo_n)))
    out = []
    for k in range(n_inst):
        if k % 2 == 0:
            lc = max(2, 2 * int(round(target[k] / 324.0)))
            out.append(sod(seed + k, nl=12, length_cells=lc, dx=1.0 / 192.0))
        else:
            nn = max(13, int(round(target[k] ** (1.0 / 3.0))))
            out.append(sedov(n=nn, seed=seed + k))
    return out


def mlp_init(seed: int = 2511, n_in: int = 4, n_hid: int = 32) -> np.ndarray:
    """Initial parameters of the seed network as one flat float64 vector in
    the order W1 (n_hid x n_in), b1, W2 (n_hid x n_hid), b2, W3 (n_hid), b3:
    hidden weights uniform in +-sqrt(6 / fan_in) (He et al. 2015), biases and
    the output layer zero, so the untrained network outputs exactly 0."""
    def he(count, fan_in, stream):
        u = uniform01(seed, np.arange(count, dtype=np.uint64), stream)
        return (2.0 * u - 1.0) * math.sqrt(6.0 / fan_in)
    W1 = he(n_hid * n_in, n_in, 0)
    W2 = he(n_hid * n_hid, n_hid, 1)
    return np.concatenate([W1, np.zeros(n_hid), W2, np.zeros(n_hid), np.zeros(n_hid),
                           np.zeros(1)])
