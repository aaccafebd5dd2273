"""The persistent 2d inner solve (one cooperative launch per float32 inner PCG) against the
oracle and against the four-kernel inner iteration it replaces.

Mixed-precision solves are refined in double-float to the requested rtol, so both inner
forms must reach the same solution within the refinement's tolerance; at sizes the oracle's
dense solve cannot reach, the right-hand side is b = G u* for a known smooth u* (the oracle's
matrix-free operator forms it) and the solve must return u*.
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


def bump_problem(nx, ny, Lx, Ly, H=0.5, R=None, seed=0):
    """Gaussian-bump depth with a wave on it, and b = G u* for a smooth u* (the oracle's
    operator)."""
    X, Y = I.grid_2d(nx, ny, Lx, Ly)
    R = R if R is not None else min(Lx, Ly) / 8
    h = I.gaussian_bump_2d(X, Y, Lx, Ly, H, R, Lx / 2, Ly / 2)
    eta = h + 0.2 * np.exp(np.cos(2 * np.pi * X / Lx) - 1)
    gh = O.grad(h, (Lx, Ly))
    us = np.stack([0.3 * np.sin(2 * np.pi * X / Lx) * np.cos(4 * np.pi * Y / Ly),
                   0.2 * np.cos(2 * np.pi * X / Lx) + 0.1 * np.sin(2 * np.pi * Y / Ly)])
    grid = O.make_grid(2, nx, Lx, 9.81, ny=ny, Ly=Ly)
    b = O.apply_G(eta, gh, us, grid)
    return eta, gh, b, us, grid


@pytest.mark.parametrize("n,a,b", [(32, 1.0, 1.0), (64, 1.0, 20.0), (128, 1.0, 1.0)])
def test_persistent_inner_solve_matches_oracle(S, n, a, b):
    """Eq:ellipticalbump (§6.3): mixed solve with either inner form equals the oracle's
    float64 solution."""
    sgn, ctx = S
    _, _, h, eta, rhs = I.elliptical_bump_2d(n, a, b)
    gh = O.grad(h, (1.0, 1.0))
    grid = O.make_grid(2, n, 1.0, 1.0, ny=n, Ly=1.0)
    ref = O.solve_G(eta, gh, rhs, grid, rtol=1e-14, maxit=4000)[0]
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, 1.0, ny=n, Ly=1.0)])
    assert lay.form2d()[0] == 0                     # persistent by default
    for form in (0, 1):
        lay.set_form2d(form, 0)
        x = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(eta), dev(gh), dev(rhs), x, rtol=1e-12, maxit=4000,
                       prec=sgn.PREC_MIXED)[0]
        assert info["status"] == 0 and info["ratio"] <= 1e-12
        assert rel(x.cpu().numpy().reshape(2, n, n), ref) < 1e-9


@pytest.mark.parametrize("nx,ny,Lx,Ly", [(8, 8, 1.0, 1.0), (16, 8, 2.0, 1.0), (256, 64, 80.0, 20.0),
                                         (512, 512, 80.0, 80.0), (1024, 256, 80.0, 20.0),
                                         (1024, 1024, 80.0, 80.0)])
def test_persistent_equals_four_kernel_form(S, nx, ny, Lx, Ly):
    """Both inner forms refine to the same solution (within the tolerance), which is the
    known u*; the persistent form repeats bitwise (fixed-order reductions)."""
    sgn, ctx = S
    eta, gh, b, us, _ = bump_problem(nx, ny, Lx, Ly)
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, Lx, ny=ny, Ly=Ly, g=9.81)])
    out = {}
    # the four-kernel form, the persistent form (twice: bitwise repeatable), and the
    # persistent form with radix-16 stages
    for form in (1, 0, 0, 2):
        lay.set_form2d(1 if form == 1 else 0, 0)
        lay.set_radix2d(16 if form == 2 else 8)
        x = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(eta), dev(gh), dev(b), x, rtol=1e-11, maxit=4000,
                       prec=sgn.PREC_MIXED)[0]
        assert info["status"] == 0 and info["ratio"] <= 1e-11, (form, info)
        if form in out:
            assert torch.equal(out[form][0], x)               # repeatable bitwise
        out[form] = (x, info)
    x1, x0, x8 = out[1][0].cpu().numpy(), out[0][0].cpu().numpy(), out[2][0].cpu().numpy()
    assert rel(x0, x1) < 1e-9 and rel(x8, x0) < 1e-9
    assert rel(x0.reshape(2, ny, nx), us) < 1e-8
    assert lay.radix2d() == 16
    lay.set_radix2d(0)                  # the default
    assert lay.radix2d() == 8
    # same method, so the inner iteration counts stay close
    i0, i1 = out[0][1]["iters"], out[1][1]["iters"]
    assert abs(i0 - i1) <= max(2, 0.1 * i1), (i0, i1)


@pytest.mark.parametrize("nx,ny,L", [(16, 16, 10.0), (64, 128, 20.0), (512, 512, 80.0),
                                     (1024, 1024, 160.0)])
def test_unit_threads_agree_and_default_follows_the_unit_count(S, nx, ny, L):
    """128 and 256 threads per unit solve to the known u* and agree within the tolerance;
    the default takes 256 when the largest phase has at most one unit per 256-thread group
    of the grid (one instance up to 512^2 on 152 SMs) and 128 otherwise (1024^2), and
    equals that choice bitwise."""
    sgn, ctx = S
    eta, gh, b, us, _ = bump_problem(nx, ny, L, L * ny / nx)
    lay = sgn.Layout(ctx, [sgn.Grid(2, nx, L, ny=ny, Ly=L * ny / nx, g=9.81)])
    out = {}
    for gt in (128, 256, 0):
        lay.set_unit_threads2d(gt)
        assert lay.unit_threads2d() == gt
        x = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(eta), dev(gh), dev(b), x, rtol=1e-11, maxit=4000,
                       prec=sgn.PREC_MIXED)[0]
        assert info["status"] == 0 and info["ratio"] <= 1e-11, (gt, info)
        out[gt] = x
    x128, x256 = out[128].cpu().numpy(), out[256].cpu().numpy()
    assert rel(x128, x256) < 1e-9
    assert rel(x256.reshape(2, ny, nx), us) < 1e-8
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    units = max(nx // 2 + 1, ny // 2)
    chosen = 256 if units <= 2 * min(sms, units) else 128
    assert torch.equal(out[0], out[chosen])
    with pytest.raises(sgn.SgnError):
        lay.set_unit_threads2d(64)
    lay.close()


def test_persistent_inner_solve_edge_cases(S):
    """A zero right-hand side, an exact warm start, too small an iteration budget and a
    non-positive depth behave as in the four-kernel form."""
    sgn, ctx = S
    n = 32
    _, _, h, eta, rhs = I.elliptical_bump_2d(n, 1.0, 1.0)
    gh = O.grad(h, (1.0, 1.0))
    lay = sgn.Layout(ctx, [sgn.Grid(2, n, 1.0, ny=n, Ly=1.0)])
    p = sgn.PREC_MIXED
    x = dev(np.ones(2 * n * n))
    info = sgn.pcg(lay, dev(eta), dev(gh), dev(np.zeros(2 * n * n)), x, prec=p)[0]
    assert info["status"] == 0 and info["iters"] == 0 and torch.all(x == 0.0)
    ref = np.linalg.solve(O.dense_G_2d(eta, gh, 1.0, 1.0), rhs.ravel())
    x = dev(ref)
    info = sgn.pcg(lay, dev(eta), dev(gh), dev(rhs), x, rtol=1e-8, prec=p)[0]
    assert info["status"] == 0 and info["iters"] == 0
    x = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    info = sgn.pcg(lay, dev(eta), dev(gh), dev(rhs), x, rtol=1e-14, maxit=2, prec=p,
                   check=False)[0]
    assert info["status"] == 5 and info["iters"] <= 3
    bad = eta.copy()
    bad[3, 5] = -0.5
    x = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    info = sgn.pcg(lay, dev(bad), dev(gh), dev(rhs), x, prec=p, check=False)[0]
    assert info["status"] == 7
    with pytest.raises(sgn.SgnError):
        lay.set_form2d(2, 0)
    with pytest.raises(sgn.SgnError):
        lay.set_form2d(0, 3)
    with pytest.raises(sgn.SgnError):
        lay.set_form2d(0, 2)             # one column per tile
    with pytest.raises(sgn.SgnError):
        lay.set_radix2d(4)


def test_autotune_2d_chooses_a_form_and_restores_the_state(S):
    """sgn_state_autotune on a 2d state times the inner-solve forms, radix plans and unit
    widths on the state's own RK4 steps, leaves one of them set, and restores the state
    bitwise; the next steps equal the same steps taken with that choice set by hand."""
    sgn, ctx = S
    n = 128
    c = I.bump2d_case(n=n, L=40.0, a=0.2, x0=10.0, H=0.5, R=3.0, dt=0.05)
    g = sgn.Grid(2, n, 40.0, g=9.81, ny=n, Ly=40.0)

    def state(lay):
        eta, u, h = dev(c["eta"]), dev(c["u"]), dev(c["h"])
        U = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
        gh = torch.zeros_like(U)
        st = sgn.State(lay, eta, U, u, h, gh)
        st.init()
        return st, eta, u

    lay = sgn.Layout(ctx, [g])
    st, eta, u = state(lay)
    eta0, u0 = eta.clone(), u.clone()
    ms = st.autotune([0.05], rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
    assert ms > 0.0
    form = lay.form2d()[0]
    radix = lay.radix2d()
    gt = lay.unit_threads2d()
    assert form in (0, 1) and radix in (8, 16) and gt in (0, 128, 256)
    assert torch.equal(eta, eta0) and torch.equal(u, u0)
    st.rk4(0.05, 3, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
    lay2 = sgn.Layout(ctx, [g])
    lay2.set_form2d(form, 0)
    lay2.set_radix2d(radix)
    lay2.set_unit_threads2d(gt)
    st2, eta2, u2 = state(lay2)
    st2.rk4(0.05, 3, rtol=1e-10, maxit=4000, prec=sgn.PREC_MIXED)
    torch.cuda.synchronize()
    assert torch.equal(eta, eta2) and torch.equal(u, u2)
    st.close()
    st2.close()


def test_layouts_of_other_sizes_leave_a_larger_layout_usable(S):
    """A layout created after a larger one (a smaller persistent-kernel shared-memory need)
    must not break the larger layout's later solves: both solve to their known u*."""
    sgn, ctx = S
    big = sgn.Layout(ctx, [sgn.Grid(2, 512, 80.0, ny=512, Ly=80.0, g=9.81)])
    small = sgn.Layout(ctx, [sgn.Grid(2, 64, 20.0, ny=64, Ly=20.0, g=9.81)])
    for lay, (n, L) in ((big, (512, 80.0)), (small, (64, 20.0)), (big, (512, 80.0))):
        eta, gh, b, us, _ = bump_problem(n, n, L, L)
        x = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(eta), dev(gh), dev(b), x, rtol=1e-10, maxit=4000,
                       prec=sgn.PREC_MIXED)[0]
        assert info["status"] == 0 and info["ratio"] <= 1e-10
        assert rel(x.cpu().numpy().reshape(2, n, n), us) < 1e-7
    big.close()
    small.close()
