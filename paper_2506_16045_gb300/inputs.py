"""Seeded synthetic inputs for the SGN constraint solve and time stepping.

This module only *generates* problem data (grids, bathymetry, initial surfaces and
velocities, right-hand sides, ensemble parameters).  It holds none of the method's
arithmetic: no derivative, no operator, no solve.  Both the CUDA path and the CPU oracle
receive the arrays produced here and compute everything else their own way.

Profiles follow the paper:
  * solitary wave, §6 (ExSleta / ExSlu): eta = h0 + a sech^2(gamma xi), u = c (eta - h0)/eta,
    c = sqrt(g (h0 + a)), gamma = sqrt(3a) / (2 h0 sqrt(h0 + a)); with g = 1 this is the
    paper's c = sqrt(h0 + a), gamma = sqrt(3a)/(2 h0 c).  On a periodic domain the profile is
    summed over periodic images so that it is smooth and periodic.
  * 1d preconditioner test problem, §6.2 (Eq:Testproblem, Eq:Testproblem1_var).
  * 2d elliptical bump, §6.3 (Eq:ellipticalbump).
  * underwater shelf, §6.4 Test 2: the paper does not give the shelf's formula, so a smooth
    periodic tanh plateau stands in for it (depth 1 -> r over a length W, ramps of width w).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "grid_1d", "grid_2d", "solitary_wave_1d", "solitary_wave_2d", "shelf_1d",
    "gaussian_bump_2d", "testproblem_1d", "elliptical_bump_2d", "Instance1d",
    "ensemble_1d", "shelf_case", "SHELF_DT", "solitary_case", "bump2d_case",
]


def grid_1d(n: int, L: float) -> np.ndarray:
    """x_j = j L / n, j = 0..n-1 (§6.1)."""
    return np.arange(n, dtype=np.float64) * (L / n)


def grid_2d(nx: int, ny: int, Lx: float, Ly: float):
    """Row-major [ny, nx] coordinate planes (X, Y)."""
    x = np.arange(nx, dtype=np.float64) * (Lx / nx)
    y = np.arange(ny, dtype=np.float64) * (Ly / ny)
    Y, X = np.meshgrid(y, x, indexing="ij")
    return X, Y


def _sech2(z):
    # sech^2 z = 4 e^{-2|z|} / (1 + e^{-2|z|})^2, written to avoid overflow for large |z|
    e = np.exp(-2.0 * np.abs(z))
    return 4.0 * e / (1.0 + e) ** 2


def solitary_params(h0: float, a: float, g: float):
    c = math.sqrt(g * (h0 + a))
    gamma = math.sqrt(3.0 * a) / (2.0 * h0 * math.sqrt(h0 + a))
    return c, gamma


def solitary_wave_1d(x, L, h0, a, x0, g, t=0.0, images=3):
    """Right-moving solitary wave crest at x0 + c t, summed over periodic images."""
    c, gamma = solitary_params(h0, a, g)
    xc = x0 + c * t
    s = np.zeros_like(x)
    for m in range(-images, images + 1):
        s += _sech2(gamma * (x - xc + m * L))
    eta = h0 + a * s
    u = c * (eta - h0) / eta
    return eta, u


def solitary_wave_2d(X, Y, Lx, Ly, h0, a, x0, g, t=0.0, images=3):
    """Plane solitary wave travelling in +x (theta = 0): a 1d profile in x, constant in y."""
    c, gamma = solitary_params(h0, a, g)
    xc = x0 + c * t
    s = np.zeros_like(X)
    for m in range(-images, images + 1):
        s += _sech2(gamma * (X - xc + m * Lx))
    eta = h0 + a * s
    w = c * (eta - h0) / eta
    return eta, np.stack([w, np.zeros_like(w)])


def shelf_1d(x, L, r, xs, w=5.0, W=None, images=1):
    """Depth 1 outside, r on [xs, xs+W]; tanh ramps of width w; periodic images summed."""
    if W is None:
        W = 0.4 * L
    s = np.zeros_like(x)
    for m in range(-images, images + 1):
        s += np.tanh((x - xs + m * L) / w) - np.tanh((x - xs - W + m * L) / w)
    return 1.0 - 0.5 * (1.0 - r) * s


def gaussian_bump_2d(X, Y, Lx, Ly, H, R, xb, yb, images=1):
    """h = 1 - H exp(-|x - x_b|^2 / R^2), periodic images summed."""
    s = np.zeros_like(X)
    for mx in range(-images, images + 1):
        for my in range(-images, images + 1):
            s += np.exp(-((X - xb + mx * Lx) ** 2 + (Y - yb + my * Ly) ** 2) / R ** 2)
    return 1.0 - H * s


def testproblem_1d(n: int, eta0: float, hvar: float, sigma: float = 1.0 / 20.0):
    """Eq:Testproblem / Eq:Testproblem1_var on [0, 1): returns (x, h, eta, b)."""
    x = grid_1d(n, 1.0)
    h = 1.0 + hvar * np.exp(-((x - 0.5) ** 2) / sigma ** 2)
    eta = 1.0 + eta0 * np.cos(4.0 * np.pi * x) ** 2
    b = np.cos(4.0 * np.pi * x)
    return x, h, eta, b


def squarewave_1d(n: int, eta0: float, hvar: float = 1.0, sigma: float = 1.0 / 20.0):
    """The discontinuous depth of the coefficient comparison in §6.2: h as in
    Eq:Testproblem1_var, eta = 0.1 where |h'(x)|^2 <= 0.2 and 0.1 eta0 elsewhere (h' the
    analytic derivative of the Gaussian), b = cos(4 pi x).  Returns (x, h, eta, b)."""
    x = grid_1d(n, 1.0)
    g = np.exp(-((x - 0.5) ** 2) / sigma ** 2)
    h = 1.0 + hvar * g
    dh = -2.0 * hvar * (x - 0.5) / sigma ** 2 * g
    eta = np.where(dh ** 2 <= 0.2, 0.1, 0.1 * eta0)
    b = np.cos(4.0 * np.pi * x)
    return x, h, eta, b


def elliptical_bump_2d(n: int, a: float, b: float):
    """Eq:ellipticalbump on the unit torus, bump centred at the origin (minimum image)."""
    X, Y = grid_2d(n, n, 1.0, 1.0)
    Xc = np.where(X >= 0.5, X - 1.0, X)
    Yc = np.where(Y >= 0.5, Y - 1.0, Y)
    r = np.sqrt((a * Xc) ** 2 + (b * Yc) ** 2)
    r0 = 0.5
    h = np.where(r <= r0, 1.0 - 0.5 * np.cos(np.pi * r / (2.0 * r0)) ** 2, 1.0)
    eta = h + np.exp(np.cos(2.0 * np.pi * X)) + 0.25 * np.sin(4.0 * np.pi * Y)
    rhs = np.stack([np.cos(4.0 * np.pi * X), np.cos(4.0 * np.pi * Y)])
    return X, Y, h, eta, rhs


# --------------------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------------------

@dataclass
class Instance1d:
    """One 1d periodic SGN initial-value problem (flat or shelf bathymetry)."""
    n: int
    L: float
    g: float
    dt: float
    h: np.ndarray
    eta: np.ndarray
    u: np.ndarray
    params: dict = field(default_factory=dict)


def solitary_case(n=256, L=100.0, a=0.2, x0=25.0, g=9.81, h0=1.0, dt=0.01) -> Instance1d:
    """Flat-bottom solitary wave (L=100, n=256, a=0.2 at x=25, g=9.81, dt=0.01)."""
    x = grid_1d(n, L)
    eta, u = solitary_wave_1d(x, L, h0, a, x0, g)
    h = np.full(n, h0)
    return Instance1d(n, L, g, dt, h, eta, u, dict(a=a, x0=x0, h0=h0))


def shelf_case(n=4096, L=200.0, a=0.3, x0=40.0, r=0.5, xs=60.0, w=5.0, g=9.81,
               dt=0.004) -> Instance1d:
    """Solitary wave (a=0.3, crest at x0) on depth 1 approaching a shelf of depth r at xs."""
    x = grid_1d(n, L)
    h = shelf_1d(x, L, r, xs, w)
    eta, u = solitary_wave_1d(x, L, 1.0, a, x0, g)
    # eta = h + zeta with the wave riding on the local depth; the crest sits in depth-1 water
    eta = h + (eta - 1.0)
    return Instance1d(n, L, g, dt, h, eta, u, dict(a=a, x0=x0, r=r, xs=xs, w=w))


# Time steps of the shelf workload (N = 4096, L = 200, 2000 steps) per scheme.  AB4 runs at
# dt = 0.004 (Courant number dt sqrt(g (1 + a)) / dx = 0.29) to t = 8.  The linearly implicit
# SBDF2 step takes its remainder G - A explicitly and, like the paper's SBDF2 runs of §6.4
# (C = 0.05 against 0.2 for RK4), needs a smaller step: at dt = 0.004 its high wavenumbers
# grow until the run overflows between t = 3.2 and 4.8, while at dt = 0.002 it stays within
# 3e-4 of AB4 to t = 4 (both measured with the CPU oracle).  Further out, at dt = 0.002, the
# modes above n/3 grow (aliasing) and the run overflows before t = 8 unless it is dealiased.
SHELF_DT = {"ab4": 0.004, "sbdf2": 0.002}


def ensemble_1d(count=256, seed=2506, kmin=9, kmax=13, L=200.0, g=9.81,
                cfl=0.25, sizes=None) -> list[Instance1d]:
    """Batched ensemble: n = 2^k with k ~ U{kmin..kmax} (or n drawn uniformly from `sizes`),
    a ~ U[0.05, 0.4], shelf start x_s ~ U[0.3L, 0.7L], depth ratio r ~ U[0.4, 0.8], w = 5,
    W = 0.4L, crest 20 units before the shelf, dt = cfl * dx / sqrt(g (1 + a))."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        if sizes is None:
            n = 2 ** int(rng.integers(kmin, kmax + 1))
        else:
            n = int(sizes[int(rng.integers(0, len(sizes)))])
        a = float(rng.uniform(0.05, 0.4))
        xs = float(rng.uniform(0.3 * L, 0.7 * L))
        r = float(rng.uniform(0.4, 0.8))
        x0 = xs - 20.0
        dt = cfl * (L / n) / math.sqrt(g * (1.0 + a))
        inst = shelf_case(n=n, L=L, a=a, x0=x0, r=r, xs=xs, w=5.0, g=g, dt=dt)
        out.append(inst)
    return out


def manufactured_fields_1d(x, t, omega=10.0):
    """Test 1 of §6.4 on L = 1: h = 2 + sin 2 pi x, eta* = 2 + sin 2 pi x sin(omega t),
    u* = cos 2 pi x cos(omega t).  Returns (h, eta*, u*)."""
    s, c = np.sin(2 * np.pi * x), np.cos(2 * np.pi * x)
    return 2.0 + s, 2.0 + s * math.sin(omega * t), c * math.cos(omega * t)


def manufactured_case(n=256, omega=10.0) -> Instance1d:
    """The manufactured-solution run of §6.4 Test 1 at t = 0 (L = 1, g = 1, the paper's
    non-dimensional gravity); dt is chosen by the caller."""
    x = grid_1d(n, 1.0)
    h, eta, u = manufactured_fields_1d(x, 0.0, omega)
    return Instance1d(n, 1.0, 1.0, 0.0, h, eta, u, dict(omega=omega))


def series_forcing_1d(spec: dict, x):
    """Evaluates a forcing stored as a double Fourier series (entries [j, k, X, T, c] meaning
    c X(2 pi j x / L) T(k omega t), for "eta" and "U") on the grid x, grouped by time
    function: returns (phi_eta [K][n], phi_U [K][n], omega [K], theta [K]) with
    S(x, t) = sum_k cos(omega_k t + theta_k) phi_k(x)  (sin a = cos(a - pi/2))."""
    L, w = spec["L"], spec["omega"]
    f = {"cos": np.cos, "sin": np.sin}
    keys = sorted({(k, T) for part in ("eta", "U") for _, k, _, T, _ in spec[part]})
    phi = {part: np.zeros((len(keys), x.size)) for part in ("eta", "U")}
    for part in ("eta", "U"):
        for j, k, X, T, c in spec[part]:
            phi[part][keys.index((k, T))] += c * f[X](2 * np.pi * j * x / L)
    omega = np.array([k * w for k, _ in keys])
    theta = np.array([0.0 if T == "cos" else -np.pi / 2 for _, T in keys])
    return phi["eta"], phi["U"], omega, theta


def bump2d_case(n=512, L=80.0, a=0.2, x0=20.0, H=0.5, R=3.0, g=9.81, dt=0.02):
    """2d plane solitary wave (theta=0) approaching a Gaussian bump at the domain centre."""
    X, Y = grid_2d(n, n, L, L)
    h = gaussian_bump_2d(X, Y, L, L, H, R, L / 2, L / 2)
    eta, u = solitary_wave_2d(X, Y, L, L, 1.0, a, x0, g)
    eta = h + (eta - 1.0)
    return dict(n=n, L=L, g=g, dt=dt, h=h, eta=eta, u=u, X=X, Y=Y)
