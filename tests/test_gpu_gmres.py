"""The GMRES option (sgn_gmres) against the oracle's restarted GMRES.

Both run the same method (Arnoldi on G A^{-1} in the A^{-1} inner product, right
preconditioning, Givens rotations, restarts) with different orthogonalisation (the oracle's
modified Gram-Schmidt, the kernels' classical Gram-Schmidt twice) and summation orders, so
their step counts agree within max(1, 2%), and each solution's true residual measure
sqrt(r.A^{-1}r) / sqrt(b.A^{-1}b), taken with the oracle's own operators, is within rtol
(1.5 rtol: the rounding of that residual).  The solve is float64 throughout.
"""
import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2506_16045_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def ratio_Ainv(eta, gh, x, b, grid, c):
    r = b - O.apply_G(eta, gh, x, grid)
    Ai = lambda v: O.apply_Ainv(v, c["sigma"], c["alpha"], grid)
    return float(np.sqrt(np.vdot(r, Ai(r)) / np.vdot(b, Ai(b))))


def same_count(got, ref):
    return abs(got - ref) <= max(1, ref // 50)


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
    return torch.as_tensor(np.ascontiguousarray(x).ravel(), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def pack(arrs):
    return np.concatenate([np.asarray(a, dtype=np.float64) for a in arrs])


RAGGED = [(8, 1.0), (64, 1.0), (256, 1.0), (1024, 1.0), (4096, 1.0), (8192, 1.0), (16384, 1.0),
          (512, 1.0)]


def cases_1d():
    out = []
    for i, (n, L) in enumerate(RAGGED):
        eta0, hvar = (0.5, 1.0, 4.0)[i % 3], (1.0, 2.0)[i % 2]
        _, h, eta, b = I.testproblem_1d(n, eta0, hvar)
        out.append((n, L, h, eta, O.deriv(h, L), b))
    return out


@pytest.mark.parametrize("restart", [30, 8])
def test_gmres_1d_ragged_batch_matches_oracle(S, restart):
    """Eq:Testproblem over the sweep's depth contrasts, n = 8 .. 16384 in one layout."""
    sgn, ctx = S
    cs = cases_1d()
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, L) for n, L, *_ in cs])
    x = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
    info = sgn.gmres(lay, dev(pack([c[3] for c in cs])), dev(pack([c[4] for c in cs])),
                     dev(pack([c[5] for c in cs])), x, rtol=1e-10, restart=restart, maxit=4000)
    xs = host(x)
    offs = lay.offsets
    for i, (n, L, h, eta, hx, b) in enumerate(cs):
        grid = O.make_grid(1, n, L, 1.0)
        _, steps, ratio, cycles, _ = O.gmres_G(eta, hx, b, grid, rtol=1e-10, restart=restart,
                                               maxit=4000)
        got = info[i]
        assert got["status"] == 0 and got["ratio"] <= 1e-10, (n, got)
        # short restarts make the count more sensitive to rounding: each cycle starts from
        # the previous cycle's rounded solution, and GMRES(8) here takes up to 20 cycles
        slack = max(1, steps // 50) if cycles <= 2 else max(2, steps // 20)
        assert abs(got["iters"] - steps) <= slack, (n, got, steps)
        xi = xs[offs[i]:offs[i + 1]]
        ref, _, _, c = O.solve_G(eta, hx, b, grid, rtol=1e-14, maxit=5000)
        assert ratio_Ainv(eta, hx, xi, b, grid, c) <= 1.5e-10, n
        assert rel(xi, ref) <= 1e-10 * np.sqrt(c["kappa_ub"]) * 1e3, n


def test_gmres_batch_equals_alone_bitwise(S):
    """Chunks never straddle instances and partial sums are taken in a fixed order, so an
    instance's solve does not depend on the rest of the batch."""
    sgn, ctx = S
    cs = cases_1d()[:6]
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, L) for n, L, *_ in cs])
    x = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
    info = sgn.gmres(lay, dev(pack([c[3] for c in cs])), dev(pack([c[4] for c in cs])),
                     dev(pack([c[5] for c in cs])), x, rtol=1e-11, restart=20, maxit=4000)
    xs = host(x)
    for i, (n, L, h, eta, hx, b) in enumerate(cs):
        l1 = sgn.Layout(ctx, [sgn.Grid(1, n, L)])
        x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
        i1 = sgn.gmres(l1, dev(eta), dev(hx), dev(b), x1, rtol=1e-11, restart=20, maxit=4000)
        assert np.array_equal(host(x1), xs[lay.offsets[i]:lay.offsets[i + 1]])
        assert i1[0]["iters"] == info[i]["iters"]


@pytest.mark.parametrize("n,a,b", [(64, 1.0, 1.0), (128, 1.0, 20.0)])
def test_gmres_2d_elliptical_bump(S, n, a, b):
    """Eq:ellipticalbump: steps against the oracle, true residual, and the PCG solution."""
    sgn, ctx = S
    grid = O.make_grid(2, n, 1.0, 1.0, ny=n, Ly=1.0)
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, 1.0, ny=n, Ly=1.0)])
    _, _, h, eta, rhs = I.elliptical_bump_2d(n, a, b)
    gh = O.grad(h, (1.0, 1.0))
    _, steps, _, _, c = O.gmres_G(eta, gh, rhs, grid, rtol=1e-10, restart=40, maxit=4000)
    x = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    info = sgn.gmres(lay, dev(eta), dev(gh), dev(rhs), x, rtol=1e-10, restart=40, maxit=4000)[0]
    assert info["status"] == 0 and info["ratio"] <= 1e-10
    assert same_count(info["iters"], steps), (info, steps)
    xg = host(x).reshape(2, n, n)
    assert ratio_Ainv(eta, gh, xg, rhs, grid, c) <= 1.5e-10
    ref, _, _, _ = O.solve_G(eta, gh, rhs, grid, rtol=1e-14, maxit=5000)
    assert rel(xg, ref) <= 1e-10 * np.sqrt(c["kappa_ub"]) * 1e3


def test_gmres_edge_cases(S):
    sgn, ctx = S
    n = 256
    _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
    hx = O.deriv(h, 1.0)
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0), sgn.Grid(1, 64, 1.0)])
    _, h2, eta2, b2 = I.testproblem_1d(64, 4.0, 1.0)
    hx2 = O.deriv(h2, 1.0)
    E, HX = dev(pack([eta, eta2])), dev(pack([hx, hx2]))
    # b = 0 in one instance: x = 0 there in 0 steps, the other solves normally
    x = torch.full((n + 64,), 3.0, dtype=torch.float64, device="cuda")
    info = sgn.gmres(lay, E, HX, dev(pack([np.zeros(n), b2])), x, rtol=1e-10)
    assert info[0]["iters"] == 0 and info[0]["status"] == 0 and not host(x)[:n].any()
    assert info[1]["status"] == 0 and info[1]["iters"] > 0
    # an exact initial guess: no steps
    x0 = O.solve_G(eta, hx, b, O.make_grid(1, n, 1.0, 1.0), rtol=1e-15, maxit=5000)[0]
    l1 = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    xg = dev(x0)
    i1 = sgn.gmres(l1, dev(eta), dev(hx), dev(b), xg, rtol=1e-8)[0]
    assert i1["iters"] == 0 and i1["status"] == 0
    # maxit reached: NOT_CONVERGED, reported per instance and as the call's status
    xg = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(sgn.SgnError) as e:
        sgn.gmres(l1, dev(eta), dev(hx), dev(b), xg, rtol=1e-12, restart=5, maxit=7)
    assert e.value.status == 5
    i2 = sgn.gmres(l1, dev(eta), dev(hx), dev(b), xg.zero_(), rtol=1e-12, restart=5, maxit=7,
                   check=False)[0]
    assert i2["status"] == 5 and i2["iters"] == 7 and i2["cycles"] == 2
    # GMRES(1) still converges (slowly) on this SPD system
    i3 = sgn.gmres(l1, dev(eta), dev(hx), dev(b), xg.zero_(), rtol=1e-6, restart=1, maxit=4000)[0]
    assert i3["status"] == 0 and i3["cycles"] == i3["iters"]
    # arguments
    for kw in (dict(restart=0), dict(restart=65), dict(rtol=0.0), dict(maxit=-1)):
        with pytest.raises(sgn.SgnError) as e:
            sgn.gmres(l1, dev(eta), dev(hx), dev(b), xg, **kw)
        assert e.value.status == 1
    # a non-positive depth finishes that instance with its status
    bad = eta.copy()
    bad[3] = -0.1
    with pytest.raises(sgn.SgnError) as e:
        sgn.gmres(l1, dev(bad), dev(hx), dev(b), xg.zero_(), rtol=1e-10)
    assert e.value.status == 7


def test_gmres_given_coefficients_and_replacement(S):
    """Caller-provided coefficients (here the replacement ones of §4) drive the preconditioner
    as in sgn_pcg: the step count follows the oracle's GMRES with the same A."""
    sgn, ctx = S
    n = 512
    _, h, eta, b = I.squarewave_1d(n, 0.25)
    hx = O.deriv(h, 1.0)
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    P = sgn.precond_coeffs(lay, dev(eta), dev(hx), kind=sgn.COEF_REPLACEMENT)
    _, steps, _, _, _ = O.gmres_G(eta, hx, b, O.make_grid(1, n, 1.0, 1.0), rtol=1e-10,
                                  restart=30, maxit=4000, kind="replacement")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = sgn.gmres(lay, dev(eta), dev(hx), dev(b), x, rtol=1e-10, restart=30, maxit=4000,
                     P=P)[0]
    assert info["status"] == 0 and same_count(info["iters"], steps), (info, steps)
