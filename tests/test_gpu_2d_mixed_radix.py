"""2d grids with a side that is not a power of two (n = 2^a 3^b 5^c; the §6.1 grids at sizes
such as 384 x 240) on the generic kernels (full complex spectra, mixed-radix row and column
passes, solves as one cached graph), against the oracle: gradient, G, the preconditioner, PCG in
both precisions, GMRES, the right-hand side and the RK4 / Adams-Bashforth steppers.

Tolerances as for the power-of-two 2d path: float64 operators <= 1e-12 relative L2, solves
to 1e-9 of the oracle's solution, mixed RK4 within 1e-6 of float64.
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


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def problem(nx, ny, Lx, Ly, seed=0, H=0.4):
    """Depth over a Gaussian bump (placed by the seed), a wave on it, a smooth velocity u*
    and b = G u* from the oracle's operator."""
    rng = np.random.default_rng(seed)
    X, Y = I.grid_2d(nx, ny, Lx, Ly)
    h = I.gaussian_bump_2d(X, Y, Lx, Ly, H, min(Lx, Ly) / 8, rng.uniform(0.3, 0.7) * Lx,
                           rng.uniform(0.3, 0.7) * Ly)
    eta = h + 0.2 * np.exp(np.cos(2 * np.pi * X / Lx) - 1)
    gh = O.grad(h, (Lx, Ly))
    us = np.stack([0.3 * np.sin(2 * np.pi * X / Lx) * np.cos(4 * np.pi * Y / Ly),
                   0.2 * np.cos(2 * np.pi * X / Lx) + 0.1 * np.sin(2 * np.pi * Y / Ly)])
    grid = O.make_grid(2, nx, Lx, 9.81, ny=ny, Ly=Ly)
    b = O.apply_G(eta, gh, us, grid)
    return h, eta, gh, us, b, grid


GRIDS = [(384, 240, 80.0, 50.0), (96, 96, 20.0, 20.0), (120, 64, 30.0, 16.0),
         (30, 24, 3.0, 2.4), (64, 90, 16.0, 22.5)]


@pytest.mark.parametrize("nx,ny,Lx,Ly", GRIDS)
def test_generic_2d_operators_match_oracle(S, nx, ny, Lx, Ly):
    sgn, ctx = S
    h, eta, gh, us, b, grid = problem(nx, ny, Lx, Ly)
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, Lx, ny=ny, Ly=Ly, g=9.81)])
    g = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
    sgn.spectral_grad(lay, dev(h), g)
    assert rel(host(g).reshape(2, ny, nx), gh) < 1e-12
    Gu = torch.zeros_like(g)
    sgn.apply_operator(lay, dev(eta), dev(gh), dev(us), Gu)
    assert rel(host(Gu).reshape(2, ny, nx), b) < 1e-12
    P = sgn.precond_coeffs(lay, dev(eta), dev(gh))[0]
    ref = O.precond_coeffs(eta, gh)
    for key in ("sigma", "alpha", "kappa_ub"):
        assert abs(P[key] - ref[key]) <= 1e-13 * abs(ref[key])
    z = torch.zeros_like(g)
    sgn.precond_solve(lay, [P], dev(us), z)
    assert rel(host(z).reshape(2, ny, nx), O.apply_Ainv(us, P["sigma"], P["alpha"], grid)) < 1e-12
    lay.close()


def test_generic_2d_operator_matches_dense_weak_form(S):
    """A small generic grid: the CUDA G against the oracle's dense W^T M W."""
    sgn, ctx = S
    nx, ny = 12, 10
    h, eta, gh, _, _, _ = problem(nx, ny, 1.2, 1.0, H=0.5)
    Gd = O.dense_G_2d(eta, gh, 1.2, 1.0)
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, 1.2, ny=ny, Ly=1.0)])
    for seed in range(3):
        u = np.random.default_rng(seed).standard_normal(2 * nx * ny)
        Gu = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
        sgn.apply_operator(lay, dev(eta), dev(gh), dev(u), Gu)
        assert rel(host(Gu), Gd @ u) < 1e-13
    lay.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,ny,Lx,Ly", [(96, 60, 24.0, 15.0), (384, 240, 80.0, 50.0)])
def test_generic_2d_pcg(S, prec, nx, ny, Lx, Ly):
    """The solve reaches the known u*; on the smaller grid it equals the oracle's own solve
    and (float64) takes the oracle's iteration count."""
    sgn, ctx = S
    h, eta, gh, us, b, grid = problem(nx, ny, Lx, Ly, seed=3)
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, Lx, ny=ny, Ly=Ly, g=9.81)])
    x = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
    p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
    rtol = 1e-12 if prec == "fp64" else 1e-11
    info = sgn.pcg(lay, dev(eta), dev(gh), dev(b), x, rtol=rtol, maxit=4000, prec=p)[0]
    assert info["status"] == 0 and info["ratio"] <= rtol, info
    xs = host(x).reshape(2, ny, nx)
    assert rel(xs, us) < 1e-8
    if nx * ny <= 96 * 60:
        ref, it, _, _ = O.solve_G(eta, gh, b, grid, rtol=1e-14, maxit=4000)
        assert rel(xs, ref) < 1e-9
        if prec == "fp64":
            _, it12, _, _ = O.solve_G(eta, gh, b, grid, rtol=1e-12, maxit=4000)
            assert abs(info["iters"] - it12) <= 1
        else:
            assert info["refinements"] >= 1
    lay.close()


def test_generic_2d_pcg_edge_cases(S):
    sgn, ctx = S
    nx, ny = 40, 30
    h, eta, gh, us, b, grid = problem(nx, ny, 10.0, 7.5, seed=5)
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, 10.0, ny=ny, Ly=7.5, g=9.81)])
    for prec in (sgn.PREC_FP64, sgn.PREC_MIXED):
        x = dev(np.ones(2 * nx * ny))
        info = sgn.pcg(lay, dev(eta), dev(gh), dev(np.zeros(2 * nx * ny)), x, prec=prec)[0]
        assert info["status"] == 0 and info["iters"] == 0 and np.all(host(x) == 0.0)
        ref = O.solve_G(eta, gh, b, grid, rtol=1e-15, maxit=4000)[0]
        x = dev(ref)
        info = sgn.pcg(lay, dev(eta), dev(gh), dev(b), x, rtol=1e-9, prec=prec)[0]
        assert info["status"] == 0 and info["iters"] == 0
        x = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(eta), dev(gh), dev(b), x, rtol=1e-14, maxit=2, prec=prec,
                       check=False)[0]
        assert info["status"] == 5 and info["iters"] <= 3
        bad = eta.copy()
        bad[3, 5] = -0.5
        x = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(bad), dev(gh), dev(b), x, prec=prec, check=False)[0]
        assert info["status"] == 7
    lay.close()


def test_generic_2d_gmres(S):
    sgn, ctx = S
    nx, ny = 60, 36
    h, eta, gh, us, b, grid = problem(nx, ny, 15.0, 9.0, seed=7)
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, 15.0, ny=ny, Ly=9.0, g=9.81)])
    x = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
    info = sgn.gmres(lay, dev(eta), dev(gh), dev(b), x, rtol=1e-12, restart=30, maxit=2000)[0]
    assert info["status"] == 0 and info["ratio"] <= 1e-12
    ref = O.solve_G(eta, gh, b, grid, rtol=1e-14, maxit=4000)[0]
    assert rel(host(x).reshape(2, ny, nx), ref) < 1e-9
    lay.close()


@pytest.mark.parametrize("nx,ny,Lx,Ly", [(384, 240, 80.0, 50.0), (96, 60, 24.0, 15.0)])
def test_generic_2d_rhs_matches_oracle(S, nx, ny, Lx, Ly):
    sgn, ctx = S
    h, eta, gh, us, _, _ = problem(nx, ny, Lx, Ly, seed=9)
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, Lx, ny=ny, Ly=Ly, g=9.81)])
    fe = torch.zeros(nx * ny, dtype=torch.float64, device="cuda")
    fU = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
    sgn.rhs(lay, dev(eta), dev(us), dev(h), dev(gh), fe, fU)
    re, rU = O.rhs_2d(eta, us, h, gh, Lx, Ly, 9.81)
    # the bound is the oracle's own change under a last-bit relative perturbation
    rng = np.random.default_rng(1)
    jig = lambda a: a * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], a.shape))
    pe, pU = O.rhs_2d(jig(eta), jig(us), h, jig(gh), Lx, Ly, 9.81)
    assert rel(host(fe).reshape(ny, nx), re) < max(1e-13, 20 * rel(pe, re))
    assert rel(host(fU).reshape(2, ny, nx), rU) < max(1e-13, 20 * rel(pU, rU))
    lay.close()


def _run(sgn, ctx, nx, ny, Lx, Ly, c, scheme, nsteps, prec, rtol, order=4):
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, Lx, ny=ny, Ly=Ly, g=9.81)])
    eta, u, h = dev(c["eta"]), dev(c["u"]), dev(c["h"])
    U = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
    gh = torch.zeros_like(U)
    st = sgn.State(lay, eta, U, u, h, gh)
    st.init()
    p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
    if scheme == "rk4":
        st.rk4(c["dt"], nsteps, rtol=rtol, maxit=4000, prec=p)
    else:
        st.abk(order, c["dt"], nsteps, rtol=rtol, maxit=4000, prec=p)
    stats = st.stats()
    out = host(eta).reshape(ny, nx), host(u).reshape(2, ny, nx), host(U).reshape(2, ny, nx)
    st.close()
    lay.close()
    return out, stats


def _case(nx, ny, Lx, Ly, dt):
    X, Y = I.grid_2d(nx, ny, Lx, Ly)
    h = I.gaussian_bump_2d(X, Y, Lx, Ly, 0.4, 3.0, Lx / 2, Ly / 2)
    eta, u = I.solitary_wave_2d(X, Y, Lx, Ly, 1.0, 0.2, 0.25 * Lx, 9.81)
    return {"eta": h + (eta - 1.0), "u": u, "h": h, "dt": dt}


@pytest.mark.parametrize("scheme,order", [("rk4", 0), ("ab", 3)])
def test_generic_2d_steppers_match_oracle(S, scheme, order):
    sgn, ctx = S
    nx, ny, Lx, Ly = 96, 60, 40.0, 25.0
    c = _case(nx, ny, Lx, Ly, 0.05)
    (eta, u, U), stats = _run(sgn, ctx, nx, ny, Lx, Ly, c, scheme, 6, "fp64", 1e-13, order or 4)
    ost = O.init_state(c["eta"], c["u"], c["h"], O.make_grid(2, nx, Lx, 9.81, ny=ny, Ly=Ly))
    if scheme == "rk4":
        O.run_rk4(ost, c["dt"], 6, 1e-13)
    else:
        O.run_ab(ost, order, c["dt"], 6, 1e-13)
    assert rel(eta - c["h"], ost.eta - c["h"]) < 1e-10
    assert rel(u, ost.u) < 1e-10 and rel(U, ost.U) < 1e-10
    assert stats["status"] == 0


def test_generic_2d_rk4_mixed_within_1e6_of_fp64(S):
    sgn, ctx = S
    nx, ny, Lx, Ly = 384, 240, 80.0, 50.0
    c = _case(nx, ny, Lx, Ly, 0.04)
    (e6, u6, _), s6 = _run(sgn, ctx, nx, ny, Lx, Ly, c, "rk4", 5, "fp64", 1e-12)
    (em, um, _), sm = _run(sgn, ctx, nx, ny, Lx, Ly, c, "rk4", 5, "mixed", 1e-11)
    assert s6["status"] == 0 and sm["status"] == 0
    assert rel(em - c["h"], e6 - c["h"]) < 1e-6 and rel(um, u6) < 1e-6


def test_generic_2d_rejections(S):
    sgn, ctx = S
    for nx, ny in ((14, 16), (16, 14), (2048, 64), (4, 64)):
        with pytest.raises(sgn.SgnError) as e:
            sgn.Layout(ctx, [sgn.Grid(2, nx, 1.0, ny=ny, Ly=1.0)])
        assert e.value.status == 2, (nx, ny)
    with pytest.raises(sgn.SgnError):
        sgn.Layout(ctx, [sgn.Grid(2, 96, 1.0, ny=96, Ly=1.0)] * 2)      # no generic batches
    nx, ny = 48, 36
    c = _case(nx, ny, 12.0, 9.0, 0.05)
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, 12.0, ny=ny, Ly=9.0, g=9.81)])
    with pytest.raises(sgn.SgnError):
        lay.set_form2d(1, 0)
    with pytest.raises(sgn.SgnError):
        lay.set_radix2d(8)
    eta, u, h = dev(c["eta"]), dev(c["u"]), dev(c["h"])
    U = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
    st = sgn.State(lay, eta, U, u, h, torch.zeros_like(U))
    st.init()
    with pytest.raises(sgn.SgnError):
        st.set_dealias(True)
    with pytest.raises(sgn.SgnError):
        st.linimp(0.05, 1)
    with pytest.raises(sgn.SgnError):
        st.rk4_nc(0.05, 1)
    st.close()
    lay.close()
