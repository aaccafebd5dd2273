"""GPU parity of the 2d (doubly periodic) CUDA path against the CPU oracle (C ABI).

Vector fields are packed as two planes [x components; y components] of [ny, nx] each.
"""
import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2506_16045_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def S():
    from paper_2506_16045_gb300 import sgn
    ctx = sgn.Context(0)
    yield sgn, ctx
    ctx.close()


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64).ravel(), device="cuda")


def host(t, shape):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().reshape(shape)


def fields(nx, ny, Lx, Ly, seed=0):
    rng = np.random.default_rng(seed)
    X, Y = I.grid_2d(nx, ny, Lx, Ly)
    h = I.gaussian_bump_2d(X, Y, Lx, Ly, 0.4, min(Lx, Ly) / 8, Lx / 2, Ly / 2)
    eta = h + 0.15 * np.exp(np.cos(2 * np.pi * X / Lx) - 1) + 0.05 * np.sin(4 * np.pi * Y / Ly)
    u = np.stack([0.2 * np.sin(2 * np.pi * X / Lx) * np.cos(2 * np.pi * Y / Ly),
                  0.1 * np.cos(4 * np.pi * X / Lx) + 0.05 * np.sin(2 * np.pi * Y / Ly)])
    u = u + 0.001 * rng.standard_normal(u.shape)
    return X, Y, h, eta, u


SHAPES = [(16, 8, 2.0, 1.0), (64, 64, 1.0, 1.0), (128, 32, 40.0, 10.0), (256, 256, 80.0, 80.0)]


@pytest.mark.parametrize("nx,ny,Lx,Ly", SHAPES)
def test_grad_and_operator_2d(S, nx, ny, Lx, Ly):
    sgn, ctx = S
    _, _, h, eta, u = fields(nx, ny, Lx, Ly, nx)
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, Lx, ny=ny, Ly=Ly)])
    gh = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
    sgn.spectral_grad(lay, dev(h), gh)
    ref_gh = O.grad(h, (Lx, Ly))
    assert rel(host(gh, (2, ny, nx)), ref_gh) < 1e-12
    Gu = torch.zeros_like(gh)
    sgn.apply_operator(lay, dev(eta), dev(ref_gh), dev(u), Gu)
    grid = O.make_grid(2, nx, Lx, 9.81, ny=ny, Ly=Ly)
    assert rel(host(Gu, (2, ny, nx)), O.apply_G(eta, ref_gh, u, grid)) < 1e-12


def test_operator_2d_matches_dense_weak_form(S):
    sgn, ctx = S
    nx, ny = 16, 8
    _, _, h, eta, u = fields(nx, ny, 1.0, 0.5, 3)
    gh = O.grad(h, (1.0, 0.5))
    Gd = O.dense_G_2d(eta, gh, 1.0, 0.5)
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, 1.0, ny=ny, Ly=0.5)])
    Gu = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
    sgn.apply_operator(lay, dev(eta), dev(gh), dev(u), Gu)
    assert rel(host(Gu, (2 * nx * ny,)), Gd @ u.ravel()) < 1e-13


@pytest.mark.parametrize("a,b", [(1.0, 1.0), (1.0, 20.0)])
def test_coeffs_and_precond_2d(S, a, b):
    sgn, ctx = S
    n = 64
    _, _, h, eta, rhs = I.elliptical_bump_2d(n, a, b)
    gh = O.grad(h, (1.0, 1.0))
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, 1.0, ny=n, Ly=1.0)])
    got = sgn.precond_coeffs(lay, dev(eta), dev(gh))[0]
    want = O.precond_coeffs(eta, gh)
    for key in ("sigma", "alpha", "kappa_ub"):
        assert abs(got[key] - want[key]) <= 1e-13 * abs(want[key])
    z = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    sgn.precond_solve(lay, [got], dev(rhs), z)
    ref = O.apply_Ainv(rhs, got["sigma"], got["alpha"], O.make_grid(2, n, 1.0, 1.0, ny=n, Ly=1.0))
    assert rel(host(z, (2, n, n)), ref) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,a,b", [(32, 1.0, 1.0), (64, 1.0, 20.0), (128, 1.0, 1.0)])
def test_pcg_2d_elliptical_bump(S, prec, n, a, b):
    """Eq:ellipticalbump with U = (cos 4 pi x, cos 4 pi y) (§6.3), u0 = 0."""
    sgn, ctx = S
    _, _, h, eta, rhs = I.elliptical_bump_2d(n, a, b)
    gh = O.grad(h, (1.0, 1.0))
    grid = O.make_grid(2, n, 1.0, 1.0, ny=n, Ly=1.0)
    ref, it_ref, _, _ = O.solve_G(eta, gh, rhs, grid, rtol=1e-14, maxit=4000)
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, 1.0, ny=n, Ly=1.0)])
    x = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
    info = sgn.pcg(lay, dev(eta), dev(gh), dev(rhs), x, rtol=1e-12, maxit=4000, prec=p)[0]
    assert info["status"] == 0 and info["ratio"] <= 1e-12
    assert rel(host(x, (2, n, n)), ref) < 1e-9
    if prec == "fp64":
        # hundreds of iterations on the anisotropic bump: CG's loss of orthogonality makes
        # the exact count sensitive to rounding order, so the count is compared to 2%
        _, it12, _, _ = O.solve_G(eta, gh, rhs, grid, rtol=1e-12, maxit=4000)
        assert abs(info["iters"] - it12) <= max(1, 0.02 * it12)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pcg_2d_edge_cases(S, prec):
    """The solve's decisions, taken on the device in the solve graph: a zero right-hand side
    (x = 0, no iteration), an exact warm start (no iteration), a budget too small (not
    converged, reported), a non-positive depth (reported), and given coefficients equal to
    the computed ones (bitwise the same solve)."""
    sgn, ctx = S
    n = 32
    p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
    _, _, h, eta, rhs = I.elliptical_bump_2d(n, 1.0, 1.0)
    gh = O.grad(h, (1.0, 1.0))
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, 1.0, ny=n, Ly=1.0)])
    x = dev(np.ones(2 * n * n))
    info = sgn.pcg(lay, dev(eta), dev(gh), dev(np.zeros(2 * n * n)), x, prec=p)[0]
    assert info["status"] == 0 and info["iters"] == 0 and np.all(host(x, (2 * n * n,)) == 0.0)
    ref = np.linalg.solve(O.dense_G_2d(eta, gh, 1.0, 1.0), rhs.ravel())
    x = dev(ref)
    info = sgn.pcg(lay, dev(eta), dev(gh), dev(rhs), x, rtol=1e-8, prec=p)[0]
    assert info["status"] == 0 and info["iters"] == 0
    assert rel(host(x, ref.shape), ref) < 1e-12
    x = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    info = sgn.pcg(lay, dev(eta), dev(gh), dev(rhs), x, rtol=1e-14, maxit=2, prec=p,
                   check=False)[0]
    assert info["status"] == 5 and info["iters"] <= 2 + 1        # SGN_ERR_NOT_CONVERGED
    bad = eta.copy()
    bad[3, 5] = -0.5
    x = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    info = sgn.pcg(lay, dev(bad), dev(gh), dev(rhs), x, prec=p, check=False)[0]
    assert info["status"] == 7                                    # SGN_ERR_NONPOSITIVE_DEPTH
    P = sgn.precond_coeffs(lay, dev(eta), dev(gh))
    x1 = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    x2 = torch.zeros_like(x1)
    i1 = sgn.pcg(lay, dev(eta), dev(gh), dev(rhs), x1, rtol=1e-11, prec=p)[0]
    i2 = sgn.pcg(lay, dev(eta), dev(gh), dev(rhs), x2, rtol=1e-11, prec=p, P=P)[0]
    assert i1["iters"] == i2["iters"] and torch.equal(x1, x2)
    assert rel(host(x1, ref.shape), ref) < 1e-9


def test_rhs_2d(S):
    sgn, ctx = S
    nx, ny, Lx, Ly = 64, 32, 20.0, 10.0
    _, _, h, eta, u = fields(nx, ny, Lx, Ly, 5)
    gh = O.grad(h, (Lx, Ly))
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, Lx, g=9.81, ny=ny, Ly=Ly)])
    fe = torch.zeros(nx * ny, dtype=torch.float64, device="cuda")
    fU = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
    sgn.rhs(lay, dev(eta), dev(u), dev(h), dev(gh), fe, fU)
    re, rU = O.rhs_2d(eta, u, h, gh, Lx, Ly, 9.81)
    rng = np.random.default_rng(0)
    jig = lambda a: a * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], a.shape))
    pe, pU = O.rhs_2d(jig(eta), jig(u), h, jig(gh), Lx, Ly, 9.81)
    assert rel(host(fe, (ny, nx)), re) < max(1e-13, 20 * rel(pe, re))
    assert rel(host(fU, (2, ny, nx)), rU) < max(1e-13, 20 * rel(pU, rU))


def _gpu_run_2d(sgn, ctx, c, scheme, nsteps, prec, rtol):
    n, L = c["n"], c["L"]
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, L, g=c["g"], ny=n, Ly=L)])
    eta, u, h = dev(c["eta"]), dev(c["u"]), dev(c["h"])
    U = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    gh = torch.zeros_like(U)
    st = sgn.State(lay, eta, U, u, h, gh)
    st.init()
    p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
    if scheme == "rk4":
        st.rk4(c["dt"], nsteps, rtol=rtol, prec=p)
    elif scheme == "ab2":
        st.abk(2, c["dt"], nsteps, rtol=rtol, prec=p)
    else:
        st.linimp(c["dt"], nsteps, rtol=rtol, prec=p)
    stats = st.stats()
    out = host(eta, (n, n)), host(U, (2, n, n)), host(u, (2, n, n))
    st.close()
    return out, stats


def _oracle_run_2d(c, scheme, nsteps, rtol):
    n, L = c["n"], c["L"]
    grid = O.make_grid(2, n, L, c["g"], ny=n, Ly=L)
    st = O.init_state(c["eta"], c["u"], c["h"], grid)
    if scheme == "rk4":
        O.run_rk4(st, c["dt"], nsteps, rtol)
    elif scheme == "ab2":
        O.run_ab(st, 2, c["dt"], nsteps, rtol)
    else:
        O.run_sbdf2(st, c["dt"], nsteps, rtol)
    return st


@pytest.mark.parametrize("scheme", ["rk4", "ab2", "linimp"])
def test_steppers_2d_bump_fp64(S, scheme):
    sgn, ctx = S
    c = I.bump2d_case(n=32, L=40.0, a=0.2, x0=10.0, H=0.5, R=3.0, dt=0.05)
    (eta, U, u), stats = _gpu_run_2d(sgn, ctx, c, scheme, 6, "fp64", 1e-13)
    ref = _oracle_run_2d(c, scheme, 6, 1e-13)
    assert rel(eta - c["h"], ref.eta - c["h"]) < 1e-10
    assert rel(u, ref.u) < 1e-10 and rel(U, ref.U) < 1e-10
    assert stats["status"] == 0


def test_rk4_2d_mixed_within_1e6(S):
    sgn, ctx = S
    c = I.bump2d_case(n=64, L=40.0, a=0.2, x0=10.0, H=0.5, R=3.0, dt=0.05)
    (eta, U, u), stats = _gpu_run_2d(sgn, ctx, c, "rk4", 5, "mixed", 1e-11)
    ref = _oracle_run_2d(c, "rk4", 5, 1e-13)
    assert rel(eta, ref.eta) < 1e-6 and rel(u, ref.u) < 1e-6
    assert stats["status"] == 0
