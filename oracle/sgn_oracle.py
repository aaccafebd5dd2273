"""CPU FP64 oracle for the SGN constraint solve and its time integrators.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
baseline leg may import this module.  It shares no code with the CUDA library and never
calls it; the library never calls this module.

Everything here is a plain, slow, obviously-correct restatement of the paper
(Feng, Shirokoff, Choi: "Preconditioning and Linearly Implicit Time Integration for the
Serre-Green-Naghdi Equations") in float64 numpy:

  * spectral derivative D = F^{-1}(iK)F with the n/2 wavenumber set to 0 (§6.1); the FFT
    is numpy's (a library primitive), and the dense derivative matrix is also built from
    its closed form (the textbook periodic cotangent matrix) as an independent check;
  * the constraint operator G_{eta,h} term by term from Def:G (§2.2), and its dense
    matrix W^T M W from the block form of the bilinear form B (Appendix A, Def:MatrixM);
  * the preconditioner A = sigma I - alpha grad(div) (Def:A, §4) and its inverse per
    Fourier mode (a 1x1 or 2x2 solve per mode);
  * the coefficients sigma*, alpha*, kappa_ub (Eq:FlatbathCoeff, Eq:Optcoeff,
    Eq:Optcoeffb) and the replacement coefficients (Remark "replacementcoeff", §4);
  * textbook preconditioned conjugate gradients (§3.2, Eq:PCGLinSyst), and textbook
    restarted GMRES, right-preconditioned by A in the A^{-1} inner product, as the Krylov
    option besides PCG;
  * the right-hand side of the DAE form (Eq:DAE_DSWE, §5) with the forcing F (Def:bigF);
  * RK4 (Eq:ERK, §5.1), Adams-Bashforth 2-4 (Eq:AB, Table 1, §5.2) and the linearly
    implicit SBDF2 step (Eq:MM, §5.3);
  * the manufactured solution of §6.4 Test 1 and its forcing;
  * the 2/3-rule projection used as dealiasing (§6.4, Test 2 remark), and the
    non-constraint form (Eq:dswe, Eq:MomEq) with its RK4 stepper (the remark of §5).

Readings of the paper that the code takes (each one is listed with its reason in the
design notes of the repository):
  R1  g is kept explicit: the momentum flux term is g*eta*grad(zeta); F carries no g.
  R2  RK4 stage sums start from U_n (the paper's "u_n" in Eq:ERK_uStage is a typo) and
      the final update is U_{n+1} = U_n + dt sum b_j f_U^{(j)}, followed by a solve for u_{n+1}.
  R3  the n/2 wavenumber is 0 for every derivative (§6.1).
  R4  grad h is the discrete spectral gradient D h; maxima/minima are over grid points.
  R5  the bottom is treated as flat iff max |grad h| <= 1e-12 (a slope, dimensionless).
  R6  (u.grad)^2 h is the operator u.grad applied twice: u.grad(u.grad h).
  R7  PCG stops when sqrt(r.A^{-1}r) <= rtol * sqrt(b.A^{-1}b).
  R8  time-stepping solves warm-start from the most recent velocity.
  R9  AB_s and SBDF2 take RK4 steps of the same dt for their start-up levels.
  R10 the SBDF2 preconditioner A is fixed from the initial data (§6.5).
  R18 GMRES runs in the A^{-1} inner product, so it minimises the residual measure of R7.
  R19 optional dealiasing: Orszag's 2/3 rule applied to every new time level (zeta and U
      before u is solved from them; u too in SBDF2, where it is not solved from U); in 2d the
      tensor product of the 1d projections.
  R20 the non-constraint form (Eq:dswe, the remark of §5) is advanced on (eta, u) with the
      RK4 tableau; u_t solves G u_t = M, M the u_t-free terms of Eq:MomEq.

Field layout: 1d fields are arrays [n]; 2d scalar fields are [ny, nx] (row-major, x
fastest), 2d vector fields are [2, ny, nx] (x component first).
"""
from __future__ import annotations

import math

import numpy as np

LAMBDA_PLUS = (4.0 + math.sqrt(13.0)) / 6.0   # eigenvalues of [[1, 1/2], [1/2, 1/3]] (App. A)
LAMBDA_MINUS = (4.0 - math.sqrt(13.0)) / 6.0
FLAT_SLOPE_TOL = 1e-12                         # reading R5

# Table 1 (Table:LMMCoeffs): coefficients listed for j = 0..s
AB_A = {2: (0.0, -1.0, 1.0), 3: (0.0, 0.0, -1.0, 1.0), 4: (0.0, 0.0, 0.0, -1.0, 1.0)}
AB_B = {2: (-0.5, 1.5), 3: (5.0 / 12, -16.0 / 12, 23.0 / 12),
        4: (-9.0 / 24, 37.0 / 24, -59.0 / 24, 55.0 / 24)}
SBDF2_A = (0.5, -2.0, 1.5)
SBDF2_B = (-1.0, 2.0)
SBDF2_C = (0.0, 0.0, 1.0)
RK4_A = ((), (0.5,), (0.0, 0.5), (0.0, 0.0, 1.0))
RK4_B = (1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6)


# ======================================================================================
# Spectral differentiation (§6.1)
# ======================================================================================

def wavenumbers(n: int, L: float) -> np.ndarray:
    """k_j = 2 pi j / L in FFT order (j = 0..n/2-1, -n/2..-1) with the n/2 entry set to 0."""
    j = np.fft.fftfreq(n, d=1.0 / n)
    k = 2.0 * np.pi * j / L
    if n % 2 == 0:
        k[n // 2] = 0.0
    return k


def deriv(f: np.ndarray, L: float, axis: int = -1) -> np.ndarray:
    """D f = F^{-1} (i K) F f along `axis` (§6.1)."""
    n = f.shape[axis]
    k = wavenumbers(n, L)
    shape = [1] * f.ndim
    shape[axis] = n
    fh = np.fft.fft(f, axis=axis)
    return np.real(np.fft.ifft(1j * k.reshape(shape) * fh, axis=axis))


def dx2(f, Lx):
    """x-derivative of a [ny, nx] field."""
    return deriv(f, Lx, axis=-1)


def dy2(f, Ly):
    """y-derivative of a [ny, nx] field."""
    return deriv(f, Ly, axis=-2)


def grad(h, L):
    """Spectral gradient (reading R4). 1d: [n] -> [n]; 2d: [ny,nx] -> [2,ny,nx]."""
    if h.ndim == 1:
        return deriv(h, L)
    Lx, Ly = L
    return np.stack([dx2(h, Lx), dy2(h, Ly)])


def diff_matrix_fft(n: int, L: float) -> np.ndarray:
    """Dense D built column by column from the FFT definition."""
    return np.stack([deriv(e, L) for e in np.eye(n)], axis=1)


def diff_matrix_cot(n: int, L: float) -> np.ndarray:
    """Closed form of the periodic spectral derivative for even n (Nyquist derivative 0):
    D_jl = (pi/L) (-1)^(j-l) cot(pi (j-l)/n) for j != l, and 0 on the diagonal."""
    j = np.arange(n)
    s = j[:, None] - j[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        D = (math.pi / L) * np.where(s % 2 == 0, 1.0, -1.0) / np.tan(math.pi * s / n)
    D[s == 0] = 0.0
    return D


# ======================================================================================
# The constraint operator G_{eta,h} (Def:G, §2.2)
# ======================================================================================

def apply_G_1d(eta, hx, u, L):
    """G u = eta u - (eta^3/3 u_x)_x - (eta^2/2 h_x u)_x + eta^2/2 h_x u_x + eta h_x (h_x u)."""
    d = deriv(u, L)                     # div u
    s = hx * u                          # grad h . u
    return (eta * u
            - deriv(eta ** 3 / 3.0 * d, L)
            - deriv(eta ** 2 / 2.0 * s, L)
            + eta ** 2 / 2.0 * hx * d
            + eta * hx * s)


def apply_G_2d(eta, gradh, u, Lx, Ly):
    """Def:G on the torus: u, gradh are [2, ny, nx]; grad and div are spectral."""
    hx, hy = gradh
    d = dx2(u[0], Lx) + dy2(u[1], Ly)
    s = hx * u[0] + hy * u[1]
    t1 = eta ** 3 / 3.0 * d
    t2 = eta ** 2 / 2.0 * s
    out = np.empty_like(u)
    out[0] = eta * u[0] - dx2(t1, Lx) - dx2(t2, Lx) + eta ** 2 / 2.0 * hx * d + eta * hx * s
    out[1] = eta * u[1] - dy2(t1, Ly) - dy2(t2, Ly) + eta ** 2 / 2.0 * hy * d + eta * hy * s
    return out


def apply_G(eta, gradh, u, grid):
    if grid["dim"] == 1:
        return apply_G_1d(eta, gradh, u, grid["Lx"])
    return apply_G_2d(eta, gradh, u, grid["Lx"], grid["Ly"])


def dense_G_1d(eta, hx, L):
    """G = W^T M W with W = [I; D] and M(x_j) the 2x2 matrix of Def:MatrixM in 1d
    (eta [[1 + h_x^2, eta h_x/2], [eta h_x/2, eta^2/3]]), D from the cotangent formula."""
    n = eta.size
    D = diff_matrix_cot(n, L)
    I = np.eye(n)
    W = np.vstack([I, D])
    M = np.zeros((2 * n, 2 * n))
    M[:n, :n] = np.diag(eta * (1.0 + hx ** 2))
    M[:n, n:] = np.diag(eta * eta * hx / 2.0)
    M[n:, :n] = np.diag(eta * eta * hx / 2.0)
    M[n:, n:] = np.diag(eta ** 3 / 3.0)
    return W.T @ M @ W


def dense_G_2d(eta, gradh, Lx, Ly):
    """G = W^T M W, W = [[I, 0], [0, I], [Dx, Dy]] on the flattened [ny*nx] grid, and
    M(x) = eta [[I + grad h grad h^T, eta grad h/2], [eta grad h^T/2, eta^2/3]] (Def:MatrixM)."""
    ny, nx = eta.shape
    N = nx * ny
    Dx = np.kron(np.eye(ny), diff_matrix_cot(nx, Lx))
    Dy = np.kron(diff_matrix_cot(ny, Ly), np.eye(nx))
    I = np.eye(N)
    Z = np.zeros((N, N))
    W = np.block([[I, Z], [Z, I], [Dx, Dy]])
    e = eta.ravel()
    hx = gradh[0].ravel()
    hy = gradh[1].ravel()
    M = np.zeros((3 * N, 3 * N))
    diag = np.diag
    M[:N, :N] = diag(e * (1.0 + hx * hx))
    M[:N, N:2 * N] = diag(e * hx * hy)
    M[N:2 * N, :N] = diag(e * hx * hy)
    M[N:2 * N, N:2 * N] = diag(e * (1.0 + hy * hy))
    M[:N, 2 * N:] = diag(e * e * hx / 2.0)
    M[2 * N:, :N] = diag(e * e * hx / 2.0)
    M[N:2 * N, 2 * N:] = diag(e * e * hy / 2.0)
    M[2 * N:, N:2 * N] = diag(e * e * hy / 2.0)
    M[2 * N:, 2 * N:] = diag(e ** 3 / 3.0)
    return W.T @ M @ W


def dense_A_1d(sigma, alpha, n, L):
    """A = sigma I + alpha D^T D (§6.1)."""
    D = diff_matrix_cot(n, L)
    return sigma * np.eye(n) + alpha * D.T @ D


def dense_A_2d(sigma, alpha, nx, ny, Lx, Ly):
    """A = sigma I + alpha Div^T Div with Div = [Dx, Dy] (the weak form A[u, v], §3.1)."""
    Dx = np.kron(np.eye(ny), diff_matrix_cot(nx, Lx))
    Dy = np.kron(diff_matrix_cot(ny, Ly), np.eye(nx))
    Div = np.hstack([Dx, Dy])
    return sigma * np.eye(2 * nx * ny) + alpha * Div.T @ Div


# ======================================================================================
# The preconditioner A (Def:A, §4) and its coefficients
# ======================================================================================

def precond_coeffs(eta, gradh, kind: str = "opt"):
    """sigma*, alpha*, kappa_ub from Eq:FlatbathCoeff / Eq:Optcoeff / Eq:Optcoeffb, or the
    replacement coefficients of the remark on replacing eta|grad h|^2 (§4).
    Returns dict(sigma, alpha, kappa_ub, flat, eta_min, eta_max)."""
    eta_min = float(np.min(eta))
    eta_max = float(np.max(eta))
    if eta_min <= 0.0:
        raise ValueError("eta_min <= 0: the theorem needs a positive depth")
    g2 = gradh ** 2 if gradh.ndim == eta.ndim else np.sum(gradh ** 2, axis=0)
    slope_max = float(np.sqrt(np.max(g2)))
    flat = slope_max <= FLAT_SLOPE_TOL
    ratio3 = (eta_max / eta_min) ** 3
    if flat:
        sigma = eta_max
        alpha = eta_max ** 3 / 3.0
        kappa = ratio3
    elif kind == "opt":
        sigma = float(np.max(eta + LAMBDA_PLUS * eta * g2))
        alpha = LAMBDA_PLUS * eta_max ** 3
        kappa = max(sigma / eta_min, (LAMBDA_PLUS / LAMBDA_MINUS) * ratio3)
    elif kind == "replacement":
        sigma = eta_max * (1.0 + LAMBDA_PLUS * slope_max ** 2)
        alpha = LAMBDA_PLUS * eta_max ** 3
        kappa = max((eta_max / eta_min) * (1.0 + LAMBDA_PLUS * slope_max ** 2),
                    (LAMBDA_PLUS / LAMBDA_MINUS) * ratio3)
    else:
        raise ValueError(kind)
    return dict(sigma=sigma, alpha=alpha, kappa_ub=kappa, flat=flat,
                eta_min=eta_min, eta_max=eta_max)


def apply_Ainv(r, sigma, alpha, grid):
    """z = A^{-1} r.  1d: each Fourier mode divided by sigma + alpha k^2.  2d: each mode
    solves the 2x2 system (sigma I + alpha k k^T) z_k = r_k, the symbol of sigma I - alpha grad div."""
    if grid["dim"] == 1:
        k = wavenumbers(r.size, grid["Lx"])
        return np.real(np.fft.ifft(np.fft.fft(r) / (sigma + alpha * k * k)))
    ny, nx = r.shape[1:]
    kx = wavenumbers(nx, grid["Lx"])[None, :] * np.ones((ny, 1))
    ky = wavenumbers(ny, grid["Ly"])[:, None] * np.ones((1, nx))
    rh = np.stack([np.fft.fft2(r[0]), np.fft.fft2(r[1])])
    K = np.stack([kx, ky])                                  # [2, ny, nx]
    S = sigma * np.eye(2)[:, :, None, None] + alpha * K[:, None] * K[None, :]
    Sm = np.moveaxis(S, (0, 1), (-2, -1))                   # [ny, nx, 2, 2]
    zh = np.linalg.solve(Sm, np.moveaxis(rh, 0, -1)[..., None])[..., 0]
    zh = np.moveaxis(zh, -1, 0)
    return np.stack([np.real(np.fft.ifft2(zh[0])), np.real(np.fft.ifft2(zh[1]))])


def apply_A(u, sigma, alpha, grid):
    """A u = sigma u - alpha grad(div u) with spectral derivatives."""
    if grid["dim"] == 1:
        L = grid["Lx"]
        return sigma * u - alpha * deriv(deriv(u, L), L)
    Lx, Ly = grid["Lx"], grid["Ly"]
    d = dx2(u[0], Lx) + dy2(u[1], Ly)
    return sigma * u - alpha * np.stack([dx2(d, Lx), dy2(d, Ly)])


# ======================================================================================
# Preconditioned conjugate gradients (§3.2)
# ======================================================================================

def pcg(applyG, applyPinv, b, x0=None, rtol=1e-12, maxit=1000, history=False):
    """Textbook PCG for G x = b with preconditioner P (only P-solves are needed, §3.2).
    Stops when sqrt(r.P^{-1}r) <= rtol sqrt(b.P^{-1}b) (reading R7).
    Returns (x, iterations, final ratio[, list of iterates])."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bz = applyPinv(b)
    bnorm = math.sqrt(max(float(np.vdot(b, bz)), 0.0))
    iters = [x.copy()] if history else None
    if bnorm == 0.0:
        x[...] = 0.0
        return (x, 0, 0.0, iters) if history else (x, 0, 0.0)
    r = b - applyG(x)
    z = applyPinv(r)
    rz = float(np.vdot(r, z))
    p = z.copy()
    it = 0
    while it < maxit and math.sqrt(max(rz, 0.0)) > rtol * bnorm:
        q = applyG(p)
        pq = float(np.vdot(p, q))
        a = rz / pq
        x = x + a * p
        r = r - a * q
        z = applyPinv(r)
        rz_new = float(np.vdot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        if history:
            iters.append(x.copy())
    ratio = math.sqrt(max(rz, 0.0)) / bnorm
    return (x, it, ratio, iters) if history else (x, it, ratio)


# ======================================================================================
# Restarted GMRES with right preconditioning (the Krylov option besides PCG)
# ======================================================================================

def gmres(applyG, applyPinv, b, x0=None, rtol=1e-10, restart=30, maxit=1000, history=False):
    """Restarted GMRES(m) for G x = b with right preconditioning, in the inner product
    <u, v> = u . P^{-1} v: the Arnoldi process on G P^{-1} (modified Gram-Schmidt in that
    inner product), Givens rotations for the small least-squares problem, and
    x = x0 + P^{-1} V y at the end of each cycle.  Each iterate minimises
    sqrt(r . P^{-1} r) over its Krylov space, the residual measure of the PCG stopping rule
    (reading R7); in the Euclidean norm a fine grid's residual has a rounding floor of about
    eps ||G|| (G grows like eta^3 k^2 / 3), which this norm damps.  This is the textbook
    method in a weighted inner product; the paper solves with PCG (§3.2) and prescribes no
    GMRES variant.
    Stops when sqrt(r.P^{-1}r) <= rtol sqrt(b.P^{-1}b): inside a cycle through the rotated
    right-hand side (which equals the residual measure of the current minimiser), and on
    the true residual at every restart.  `maxit` bounds the Arnoldi steps over all cycles.
    Returns (x, steps, final true ratio, cycles[, x after every step])."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = math.sqrt(max(float(np.vdot(b, applyPinv(b))), 0.0))
    hist = [] if history else None
    if bnorm == 0.0:
        x[...] = 0.0
        return (x, 0, 0.0, 0, hist) if history else (x, 0, 0.0, 0)
    m = restart
    steps = cycles = 0
    r = b - applyG(x)
    rz = applyPinv(r)
    beta = math.sqrt(max(float(np.vdot(r, rz)), 0.0))
    while beta > rtol * bnorm and steps < maxit:
        cycles += 1
        V, Z = [r / beta], [rz / beta]                  # Z_i = P^{-1} V_i
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        j = 0
        while j < m and steps < maxit:
            w = applyG(Z[j])
            t = applyPinv(w)                             # kept equal to P^{-1} w
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = float(np.vdot(w, Z[i]))        # <w, V_i> = w . P^{-1} V_i
                w = w - H[i, j] * V[i]
                t = t - H[i, j] * Z[i]
            hnext = math.sqrt(max(float(np.vdot(w, t)), 0.0))
            H[j + 1, j] = hnext
            for i in range(j):                           # earlier rotations on the new column
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j], H[j + 1, j] = den, 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            j += 1
            steps += 1
            if history:
                y = _back_substitute(H[:j, :j], gvec[:j])
                hist.append(x + sum(y[i] * Z[i] for i in range(j)))
            if abs(gvec[j]) <= rtol * bnorm or hnext == 0.0:
                break
            V.append(w / hnext)
            Z.append(t / hnext)
        y = _back_substitute(H[:j, :j], gvec[:j])
        x = x + sum(y[i] * Z[i] for i in range(j))
        r = b - applyG(x)
        rz = applyPinv(r)
        beta = math.sqrt(max(float(np.vdot(r, rz)), 0.0))
    ratio = beta / bnorm
    return (x, steps, ratio, cycles, hist) if history else (x, steps, ratio, cycles)


def _back_substitute(R, g):
    """Solves the upper-triangular R y = g."""
    k = g.size
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - float(R[i, i + 1:] @ y[i + 1:])) / R[i, i]
    return y


def gmres_G(eta, gradh, b, grid, x0=None, rtol=1e-10, restart=30, maxit=2000, kind="opt"):
    """Solve G_{eta,h} x = b by GMRES(restart) right-preconditioned with the A of §4.
    Returns (x, steps, ratio, cycles, coefficients)."""
    c = precond_coeffs(eta, gradh, kind)
    x, it, ratio, cyc = gmres(lambda v: apply_G(eta, gradh, v, grid),
                              lambda v: apply_Ainv(v, c["sigma"], c["alpha"], grid),
                              b, x0, rtol, restart, maxit)
    return x, it, ratio, cyc, c


def solve_G(eta, gradh, b, grid, x0=None, rtol=1e-12, maxit=2000, kind="opt"):
    """Solve G_{eta,h} x = b by PCG with the preconditioner A of §4."""
    c = precond_coeffs(eta, gradh, kind)
    x, it, ratio = pcg(lambda v: apply_G(eta, gradh, v, grid),
                       lambda v: apply_Ainv(v, c["sigma"], c["alpha"], grid),
                       b, x0, rtol, maxit)
    return x, it, ratio, c


def g_error(u, ustar, G_dense, b):
    """epsilon(u) = ||u - u*||_G / ||b|| in the discrete norms of §6.1 (def:discrete_Gerr);
    the grid weight Delta x cancels."""
    e = (u - ustar).ravel()
    return math.sqrt(max(float(e @ G_dense @ e), 0.0)) / float(np.linalg.norm(b.ravel()))


def generalized_eigenvalues(G_dense, A_dense):
    """Eigenvalues of G v = lambda A v (Eq:DiscreteGenEigvalue): Cholesky A = L L^T, then the
    symmetric eigenvalues of L^{-1} G L^{-T}, ascending."""
    Lc = np.linalg.cholesky(A_dense)
    Li = np.linalg.inv(Lc)
    S = Li @ G_dense @ Li.T
    return np.linalg.eigvalsh(0.5 * (S + S.T))


# ======================================================================================
# Right-hand side of the DAE (Eq:DAE_DSWE) with the forcing F (Def:bigF)
# ======================================================================================

def rhs_1d(eta, u, h, hx, L, g):
    """Returns (f_eta, f_U):
    f_eta = -(eta u)_x,  f_U = -g eta zeta_x - (eta u u)_x + F,
    F = (eta^3 Q/3 + eta^2 m d + eta^2 S/2 + eta m s)_x - h_x (eta^2 Q/2 + eta m d + eta S + m s),
    d = u_x, Q = u d_x - d^2, m = (eta u)_x, s = h_x u, S = u s_x (reading R6)."""
    zeta = eta - h
    d = deriv(u, L)
    m = deriv(eta * u, L)
    s = hx * u
    S = u * deriv(s, L)
    Q = u * deriv(d, L) - d * d
    Phi = eta ** 3 * Q / 3.0 + eta ** 2 * m * d + eta ** 2 * S / 2.0 + eta * m * s
    Psi = eta ** 2 * Q / 2.0 + eta * m * d + eta * S + m * s
    F = deriv(Phi, L) - hx * Psi
    f_eta = -m
    f_U = -g * eta * deriv(zeta, L) - deriv(eta * u * u, L) + F
    return f_eta, f_U


def rhs_nc_1d(eta, u, h, hx, L, g):
    """The non-constraint form (Eq:dswe) in 1d, with the u_t terms grouped as in Eq:MomEq:
    eta_t = -(eta u)_x and G_{eta,h} u_t = M with
      M = -eta u u_x - g eta zeta_x + (eta^3 Q/3 + eta^2 S/2)_x - h_x (eta^2 Q/2 + eta S),
    Q = u u_xx - u_x^2 (the u.grad(div u) - (div u)^2 of Eq:MomEq), S = u (h_x u)_x (reading
    R6 for (u.grad)^2 h).  Returns (f_eta, M)."""
    zeta = eta - h
    d = deriv(u, L)
    Q = u * deriv(d, L) - d * d
    S = u * deriv(hx * u, L)
    M = (-eta * u * d - g * eta * deriv(zeta, L)
         + deriv(eta ** 3 * Q / 3.0 + eta ** 2 * S / 2.0, L)
         - hx * (eta ** 2 * Q / 2.0 + eta * S))
    return -deriv(eta * u, L), M


def rhs_2d(eta, u, h, gradh, Lx, Ly, g):
    """2d form of rhs_1d: div(eta u tensor u) has components ((eta u u)_x + (eta u v)_y,
    (eta u v)_x + (eta v v)_y) (§2.2); F = grad(Phi) - grad h Psi with d = div u,
    Q = u.grad d - d^2, m = div(eta u), s = grad h . u, S = u.grad s."""
    uu, vv = u
    hx, hy = gradh
    zeta = eta - h
    d = dx2(uu, Lx) + dy2(vv, Ly)
    m = dx2(eta * uu, Lx) + dy2(eta * vv, Ly)
    s = hx * uu + hy * vv
    S = uu * dx2(s, Lx) + vv * dy2(s, Ly)
    Q = uu * dx2(d, Lx) + vv * dy2(d, Ly) - d * d
    Phi = eta ** 3 * Q / 3.0 + eta ** 2 * m * d + eta ** 2 * S / 2.0 + eta * m * s
    Psi = eta ** 2 * Q / 2.0 + eta * m * d + eta * S + m * s
    f_eta = -m
    f_U = np.empty_like(u)
    f_U[0] = (-g * eta * dx2(zeta, Lx) - dx2(eta * uu * uu, Lx) - dy2(eta * uu * vv, Ly)
              + dx2(Phi, Lx) - hx * Psi)
    f_U[1] = (-g * eta * dy2(zeta, Ly) - dx2(eta * uu * vv, Lx) - dy2(eta * vv * vv, Ly)
              + dy2(Phi, Ly) - hy * Psi)
    return f_eta, f_U


def rhs_nc_2d(eta, u, h, gradh, Lx, Ly, g):
    """2d form of rhs_nc_1d (Eq:MomEq): G u_t = M with
      M = -eta (u.grad) u - g eta grad zeta + grad(eta^3 Q/3 + eta^2 S/2)
          - grad h (eta^2 Q/2 + eta S),
    d = div u, Q = u.grad d - d^2, s = grad h . u, S = u.grad s.  Returns (f_eta, M)."""
    uu, vv = u
    hx, hy = gradh
    zeta = eta - h
    d = dx2(uu, Lx) + dy2(vv, Ly)
    s = hx * uu + hy * vv
    S = uu * dx2(s, Lx) + vv * dy2(s, Ly)
    Q = uu * dx2(d, Lx) + vv * dy2(d, Ly) - d * d
    Phi = eta ** 3 * Q / 3.0 + eta ** 2 * S / 2.0
    Psi = eta ** 2 * Q / 2.0 + eta * S
    M = np.empty_like(u)
    M[0] = (-eta * (uu * dx2(uu, Lx) + vv * dy2(uu, Ly)) - g * eta * dx2(zeta, Lx)
            + dx2(Phi, Lx) - hx * Psi)
    M[1] = (-eta * (uu * dx2(vv, Lx) + vv * dy2(vv, Ly)) - g * eta * dy2(zeta, Ly)
            + dy2(Phi, Ly) - hy * Psi)
    return -(dx2(eta * uu, Lx) + dy2(eta * vv, Ly)), M


def dGdt_2d(eta, eta_t, gradh, u, Lx, Ly):
    """d/dt (G_{eta(t),h} u) with u and h fixed (2d Def:G by the product rule):
    eta_t u - grad(eta^2 eta_t d) - grad(eta eta_t s) + eta eta_t grad h d + eta_t grad h s."""
    hx, hy = gradh
    d = dx2(u[0], Lx) + dy2(u[1], Ly)
    s = hx * u[0] + hy * u[1]
    t1 = eta ** 2 * eta_t * d
    t2 = eta * eta_t * s
    out = np.empty_like(u)
    out[0] = eta_t * u[0] - dx2(t1, Lx) - dx2(t2, Lx) + eta * eta_t * hx * d + eta_t * hx * s
    out[1] = eta_t * u[1] - dy2(t1, Ly) - dy2(t2, Ly) + eta * eta_t * hy * d + eta_t * hy * s
    return out


def rhs(eta, u, h, gradh, grid):
    if grid["dim"] == 1:
        return rhs_1d(eta, u, h, gradh, grid["Lx"], grid["g"])
    return rhs_2d(eta, u, h, gradh, grid["Lx"], grid["Ly"], grid["g"])


# ======================================================================================
# Time integration (§5)
# ======================================================================================

class State:
    """(eta, U, u) at time t plus the fixed bathymetry (h, grad h), and an optional external
    forcing: a callable t -> (S_eta, S_U) added to the right-hand side at every stage time
    (the source term of Test 1 of §6.4)."""

    def __init__(self, eta, U, u, h, gradh, grid, t=0.0, forcing=None):
        self.eta = np.array(eta, dtype=np.float64)
        self.U = np.array(U, dtype=np.float64)
        self.u = np.array(u, dtype=np.float64)
        self.h = h
        self.gradh = gradh
        self.grid = grid
        self.t = t
        self.forcing = forcing
        self.dealias = False       # 2/3-rule projection of every new level (reading R19)
        self.solves = 0
        self.iterations = 0
        # the last step's starting u and the u it returned (reading R8's first-solve guess)
        self.u_prev = None
        self.u_last = None

    def copy(self):
        s = State(self.eta, self.U, self.u, self.h, self.gradh, self.grid, self.t, self.forcing)
        s.solves, s.iterations, s.dealias = self.solves, self.iterations, self.dealias
        s.u_prev = None if self.u_prev is None else self.u_prev.copy()
        s.u_last = None if self.u_last is None else self.u_last.copy()
        return s


def dealias_1d(f):
    """Orszag's 2/3 rule on a periodic 1d field: its Fourier modes with |j| > n/3 set to zero.
    The paper reports (§6.4, Test 2) that dealiasing, there by zero padding, helps against
    the long-time instability of large solitary waves; truncation is the form used here
    (reading R19)."""
    n = f.size
    j = np.fft.fftfreq(n, d=1.0 / n)
    fh = np.fft.fft(f)
    fh[np.abs(j) > n / 3.0] = 0.0
    return np.real(np.fft.ifft(fh))


def dealias_2d(f):
    """The 2/3 rule on a periodic [ny, nx] field: modes with |jx| > nx/3 or |jy| > ny/3 set to
    zero (the tensor product of the 1d projections)."""
    ny, nx = f.shape
    jx = np.abs(np.fft.fftfreq(nx, d=1.0 / nx))
    jy = np.abs(np.fft.fftfreq(ny, d=1.0 / ny))
    keep = (jy[:, None] <= ny / 3.0) & (jx[None, :] <= nx / 3.0)
    return np.real(np.fft.ifft2(np.fft.fft2(f) * keep))


def dealias(f, grid):
    """The 2/3 rule on a scalar (1d [n], 2d [ny, nx]) or 2d vector ([2, ny, nx]) field."""
    if grid["dim"] == 1:
        return dealias_1d(f)
    if f.ndim == 3:
        return np.stack([dealias_2d(f[0]), dealias_2d(f[1])])
    return dealias_2d(f)


def _new_level(st: State, eta, U):
    """A new time level (eta, U) as the steppers keep it: with dealiasing on, zeta = eta - h and
    U are projected before anything (the solve for u, a right-hand side) is computed from it."""
    if not st.dealias:
        return eta, U
    return st.h + dealias(eta - st.h, st.grid), dealias(U, st.grid)


def make_grid(dim, nx, Lx, g, ny=1, Ly=1.0):
    return dict(dim=dim, nx=nx, ny=ny, Lx=Lx, Ly=Ly, g=g)


def init_state(eta, u, h, grid):
    """U_0 = G_{eta_0,h} u_0 with grad h = D h (reading R4)."""
    L = grid["Lx"] if grid["dim"] == 1 else (grid["Lx"], grid["Ly"])
    gradh = grad(h, L)
    U = apply_G(eta, gradh, u, grid)
    return State(eta, U, u, h, gradh, grid)


def _rhs_t(st: State, eta, u, t):
    """f(eta, u) plus the external forcing at time t (if any)."""
    a, b = rhs(eta, u, st.h, st.gradh, st.grid)
    if st.forcing is not None:
        sa, sb = st.forcing(t)
        a, b = a + sa, b + sb
    return a, b


def _step_guess(st: State, c):
    """Reading R8: the first solve of a step starts, at every point where u is still the value
    the last step returned, from u + c (u - u_prev), the linear extrapolation from that step's
    start (c = 1/2 for the RK4 stage at t + dt/2, c = 1 for the AB solve at t + dt); elsewhere
    (no history, or u changed since) from u itself."""
    u = st.u
    if st.u_last is None:
        return u.copy()
    same = u == st.u_last
    return np.where(same, u + c * (u - st.u_prev), u)


def _solve(st: State, eta, U, x0, rtol, maxit):
    x, it, _, _ = solve_G(eta, st.gradh, U, st.grid, x0=x0, rtol=rtol, maxit=maxit)
    st.solves += 1
    st.iterations += it
    return x


def rk4_step(st: State, dt, rtol=1e-12, maxit=2000):
    """One classical RK4 step of Eq:ERK with one constraint solve per stage 2..4 and one
    for u_{n+1} (readings R2, R8: the stage at c = 1/2 starts from the extrapolated guess of
    _step_guess, the stage at c = 1 from 2 u^(3) - u_n, the others from the previous
    stage's u)."""
    eta_n, U_n, u_n = st.eta, st.U, st.u
    fe, fU = [], []
    eta_i, U_i, u_i = eta_n, U_n, u_n
    for i in range(4):
        if i > 0:
            eta_i = eta_n + dt * sum(RK4_A[i][j] * fe[j] for j in range(i))
            U_i = U_n + dt * sum(RK4_A[i][j] * fU[j] for j in range(i))
            if i == 1:
                x0 = _step_guess(st, 0.5)
            elif i == 3:
                x0 = 2.0 * u_i - u_n
            else:
                x0 = u_i
            u_i = _solve(st, eta_i, U_i, x0, rtol, maxit)
        a, b = _rhs_t(st, eta_i, u_i, st.t + dt * sum(RK4_A[i]))
        fe.append(a)
        fU.append(b)
    st.eta, st.U = _new_level(st, eta_n + dt * sum(RK4_B[j] * fe[j] for j in range(4)),
                              U_n + dt * sum(RK4_B[j] * fU[j] for j in range(4)))
    st.u = _solve(st, st.eta, st.U, u_i, rtol, maxit)
    st.u_prev, st.u_last = u_n.copy(), st.u.copy()
    st.t += dt
    return st


def rk4_nc_step(st: State, dt, rtol=1e-12, maxit=2000):
    """One RK4 step (Eq:ERK tableau) of the non-constraint form on (eta, u) (the remark of §5
    that the same time discretisations apply to Eq:dswe): each stage takes
    k = (f_eta, u_t) with G_{eta_i,h} u_t = M(eta_i, u_i) solved by PCG (warm start from the
    previous stage's u_t; stage 4 from 2 u_t^(3) - u_t^(1), as R8's stage-4 start).  U = G u is refreshed at the end so the state stays consistent.
    1d and 2d, without forcing or dealiasing."""
    grid = st.grid
    if st.forcing is not None or st.dealias:
        raise ValueError("the non-constraint stepper takes no forcing or dealiasing")
    g = grid["g"]
    if grid["dim"] == 1:
        rhs_nc = lambda e, v: rhs_nc_1d(e, v, st.h, st.gradh, grid["Lx"], g)
    else:
        rhs_nc = lambda e, v: rhs_nc_2d(e, v, st.h, st.gradh, grid["Lx"], grid["Ly"], g)
    eta_n, u_n = st.eta, st.u
    fe, ut = [], []
    ut_prev = getattr(st, "ut", np.zeros_like(u_n))
    for i in range(4):
        eta_i = eta_n + dt * sum(RK4_A[i][j] * fe[j] for j in range(i))
        u_i = u_n + dt * sum(RK4_A[i][j] * ut[j] for j in range(i))
        f_eta, M = rhs_nc(eta_i, u_i)
        if i == 3:                       # c = 1: extrapolate from c = 0 and c = 1/2
            ut_prev = 2.0 * ut[2] - ut[0]
        ut_prev = _solve(st, eta_i, M, ut_prev, rtol, maxit)
        fe.append(f_eta)
        ut.append(ut_prev)
    st.eta = eta_n + dt * sum(RK4_B[j] * fe[j] for j in range(4))
    st.u = u_n + dt * sum(RK4_B[j] * ut[j] for j in range(4))
    st.U = apply_G(st.eta, st.gradh, st.u, grid)
    st.ut = ut_prev
    st.t += dt
    return st


def run_rk4_nc(st: State, dt, nsteps, rtol=1e-12):
    for _ in range(nsteps):
        rk4_nc_step(st, dt, rtol)
    return st


def run_rk4(st: State, dt, nsteps, rtol=1e-12):
    for _ in range(nsteps):
        rk4_step(st, dt, rtol)
    return st


def run_ab(st: State, order, dt, nsteps, rtol=1e-12):
    """Adams-Bashforth of order s (Eq:AB, Table 1): w_{n+s} = w_{n+s-1} + dt sum_j b_j f_{n+j},
    then G_{eta_{n+s}} u_{n+s} = U_{n+s}.  The first s-1 steps are RK4 (reading R9)."""
    s = order
    b = AB_B[s]
    hist = [_rhs_t(st, st.eta, st.u, st.t)]
    done = 0
    while done < min(s - 1, nsteps):
        rk4_step(st, dt, rtol)
        hist.append(_rhs_t(st, st.eta, st.u, st.t))
        done += 1
    while done < nsteps:
        fe = sum(b[j] * hist[j][0] for j in range(s))
        fU = sum(b[j] * hist[j][1] for j in range(s))
        st.eta, st.U = _new_level(st, st.eta + dt * fe, st.U + dt * fU)
        u_n = st.u
        st.u = _solve(st, st.eta, st.U, _step_guess(st, 1.0), rtol, 2000)
        st.u_prev, st.u_last = u_n.copy(), st.u.copy()
        st.t += dt
        done += 1
        hist = hist[1:] + [_rhs_t(st, st.eta, st.u, st.t)]
    return st


def run_sbdf2(st: State, dt, nsteps, rtol=1e-12, coef_scale=1.0):
    """Linearly implicit SBDF2 (Eq:MM with the SBDF2 row of Table 1):
      (3/2 w_{n+2} - 2 w_{n+1} + 1/2 w_n)/dt = 2 f_{n+1} - f_n,
      A u_{n+2} = 2 (A u_{n+1} - G_{n+1} u_{n+1} + U_{n+1}) - (A u_n - G_n u_n + U_n),
    with A fixed from the initial data (reading R10, optionally scaled by coef_scale).
    The first step is RK4 (reading R9)."""
    c = precond_coeffs(st.eta, st.gradh)
    sigma, alpha = coef_scale * c["sigma"], coef_scale * c["alpha"]
    grid = st.grid
    if nsteps <= 0:
        return st
    prev = (st.eta.copy(), st.U.copy(), st.u.copy())
    f_prev = _rhs_t(st, st.eta, st.u, st.t)
    rk4_step(st, dt, rtol)
    done = 1
    while done < nsteps:
        eta0, U0, u0 = prev
        f_cur = _rhs_t(st, st.eta, st.u, st.t)
        eta2 = (4.0 * st.eta - eta0 + 2.0 * dt * (2.0 * f_cur[0] - f_prev[0])) / 3.0
        U2 = (4.0 * st.U - U0 + 2.0 * dt * (2.0 * f_cur[1] - f_prev[1])) / 3.0
        res1 = apply_A(st.u, sigma, alpha, grid) - apply_G(st.eta, st.gradh, st.u, grid) + st.U
        res0 = apply_A(u0, sigma, alpha, grid) - apply_G(eta0, st.gradh, u0, grid) + U0
        u2 = apply_Ainv(2.0 * res1 - res0, sigma, alpha, grid)
        eta2, U2 = _new_level(st, eta2, U2)
        if st.dealias:
            u2 = dealias(u2, grid)     # u is not solved from U here: it is projected too
        prev = (st.eta, st.U, st.u)
        f_prev = f_cur
        st.eta, st.U, st.u = eta2, U2, u2
        st.t += dt
        done += 1
    return st


# ======================================================================================
# Manufactured solution (Test 1 of §6.4)
# ======================================================================================

def manufactured_1d(x, t, omega=10.0):
    """Test 1 of §6.4 on L = 1: h = 2 + sin 2 pi x, eta* = 2 + sin 2 pi x sin(omega t),
    u* = cos 2 pi x cos(omega t).  Returns (h, eta*, u*, d eta*/dt, d u*/dt)."""
    s, c = np.sin(2 * np.pi * x), np.cos(2 * np.pi * x)
    h = 2.0 + s
    eta = 2.0 + s * math.sin(omega * t)
    u = c * math.cos(omega * t)
    return h, eta, u, omega * s * math.cos(omega * t), -omega * c * math.sin(omega * t)


def dGdt_1d(eta, eta_t, hx, u, u_t, L):
    """d/dt (G_{eta(t),h} u(t)) with h fixed: Def:G (1d) differentiated by the product rule,
    G_eta u_t + eta_t u - (eta^2 eta_t u_x)_x - (eta eta_t h_x u)_x + eta eta_t h_x u_x
    + eta_t h_x^2 u."""
    d = deriv(u, L)
    return (apply_G_1d(eta, hx, u_t, L) + eta_t * u - deriv(eta ** 2 * eta_t * d, L)
            - deriv(eta * eta_t * hx * u, L) + eta * eta_t * hx * d + eta_t * hx ** 2 * u)


def manufactured_forcing_1d(x, t, L, g, omega=10.0):
    """The source (S_eta, S_U) that makes (eta*, u*) solve the DAE form (Eq:DAE_DSWE) with
    U* = G_{eta*,h} u*: S_eta = d eta*/dt - f_eta(eta*, u*), S_U = dU*/dt - f_U(eta*, u*)."""
    h, eta, u, eta_t, u_t = manufactured_1d(x, t, omega)
    hx = deriv(h, L)
    fe, fU = rhs_1d(eta, u, h, hx, L, g)
    return eta_t - fe, dGdt_1d(eta, eta_t, hx, u, u_t, L) - fU


# ======================================================================================
# Diagnostics
# ======================================================================================

def mass(eta, h, cell):
    """m = integral of zeta (Remark rmk:dswe_as_constraint)."""
    return float(np.sum(eta - h)) * cell


def energy(st: State):
    """E = 1/2 integral [g zeta^2 + u . G u]; on a flat bottom u.Gu = eta|u|^2 + eta^3 (div u)^2/3
    (Remark rmk:dswe_as_constraint with g restored)."""
    grid = st.grid
    cell = grid["Lx"] / grid["nx"] * (1.0 if grid["dim"] == 1 else grid["Ly"] / grid["ny"])
    zeta = st.eta - st.h
    Gu = apply_G(st.eta, st.gradh, st.u, grid)
    return 0.5 * cell * (grid["g"] * float(np.sum(zeta ** 2)) + float(np.sum(st.u * Gu)))


def sbdf2_zero_stability_growth(G_dense, A_dense, nsteps=200, seed=0):
    """Iterate the homogeneous dt = 0 recurrence Eq:ZeroS3 for SBDF2,
    A p_{n+2} = 2 (A - G) p_{n+1} - (A - G) p_n, and return max |p_n| / |p_0|."""
    rng = np.random.default_rng(seed)
    m = G_dense.shape[0]
    p0 = rng.standard_normal(m)
    p1 = rng.standard_normal(m)
    B = A_dense - G_dense
    Ainv = np.linalg.inv(A_dense)
    n0 = max(np.linalg.norm(p0), np.linalg.norm(p1))
    growth = 1.0
    for _ in range(nsteps):
        p2 = Ainv @ (2.0 * B @ p1 - B @ p0)
        p0, p1 = p1, p2
        growth = max(growth, np.linalg.norm(p2) / n0)
    return growth
