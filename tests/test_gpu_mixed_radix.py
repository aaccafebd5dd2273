"""1d sizes that are not powers of two, n = 2^a 3^b 5^c (the grids of §6.1 at n = 96, 384,
1536, 6144, 12288, ...), on the generic kernels (mixed-radix transforms in shared memory, or
in global memory above n = 6144), against
the oracle: gradient, G, the preconditioner, PCG in both precisions, GMRES, the right-hand
side and the RK4 / Adams-Bashforth steppers, alone and in ragged batches with powers of two.

Tolerances as for the power-of-two path: float64 operators <= 1e-12 relative L2, solves to
1e-10 of the oracle's solution, the mixed solve to 1e-9, mixed RK4 within 1e-6 of float64.
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
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def pack(arrs):
    return np.concatenate([np.asarray(a, dtype=np.float64) for a in arrs])


def unpack(v, offs):
    return [v[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]


# generic sizes (every radix: 2, 4, 8, 3, 5), with powers of two mixed in
RAGGED = [(96, 80.0), (384, 200.0), (1536, 200.0), (6144, 400.0), (6, 1.0), (30, 5.0),
          (120, 10.0), (3000, 300.0), (64, 7.5), (512, 3.0), (360, 36.0), (2400, 100.0),
          (12288, 800.0), (15360, 900.0)]


def fields(n, L, seed):
    """Depth over a smooth shelf with a trough (placed by the seed), a bump of water on it
    and a smooth velocity."""
    rng = np.random.default_rng(seed)
    x = I.grid_1d(n, L)
    xs = rng.uniform(0.4, 0.6) * L
    h = 1.0 - 0.4 / (1.0 + np.exp(-(x - xs) / (0.05 * L)))
    h = h + 0.3 * np.exp(-((x - 0.25 * L) / (0.1 * L)) ** 2)
    eta = h + rng.uniform(0.1, 0.3) * np.exp(-((x - 0.6 * L) / (0.08 * L)) ** 2)
    u = 0.3 * np.sin(2 * np.pi * x / L) + 0.05 * np.cos(6 * np.pi * x / L)
    return h, eta, u


def test_generic_gradient_operator_and_preconditioner(S):
    sgn, ctx = S
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, L) for n, L in RAGGED])
    F = [fields(n, L, i) for i, (n, L) in enumerate(RAGGED)]
    h = dev(pack([f[0] for f in F]))
    gh = torch.zeros_like(h)
    sgn.spectral_grad(lay, h, gh)
    hxs = unpack(host(gh), lay.offsets)
    for (n, L), f, g in zip(RAGGED, F, hxs):
        assert rel(g, O.deriv(f[0], L)) < 1e-12, n
    eta, u = dev(pack([f[1] for f in F])), dev(pack([f[2] for f in F]))
    Gu = torch.zeros_like(u)
    sgn.apply_operator(lay, eta, gh, u, Gu)
    for (n, L), f, hx, g in zip(RAGGED, F, hxs, unpack(host(Gu), lay.offsets)):
        assert rel(g, O.apply_G_1d(f[1], hx, f[2], L)) < 1e-12, n
    P = sgn.precond_coeffs(lay, eta, gh)
    for (n, L), f, hx, p in zip(RAGGED, F, hxs, P):
        w = O.precond_coeffs(f[1], hx)
        for key in ("sigma", "alpha", "kappa_ub"):
            assert abs(p[key] - w[key]) <= 1e-14 * abs(w[key]), (n, key)
    z = torch.zeros_like(u)
    sgn.precond_solve(lay, P, u, z)
    for (n, L), f, p, zi in zip(RAGGED, F, P, unpack(host(z), lay.offsets)):
        ref = O.apply_Ainv(f[2], p["sigma"], p["alpha"], O.make_grid(1, n, L, 1.0))
        assert rel(zi, ref) < 1e-12, n


@pytest.mark.parametrize("n", [6, 24, 40, 90])
def test_generic_operator_matches_dense_weak_form(S, n):
    """Small generic n: the CUDA G against the oracle's dense W^T M W with the cotangent D."""
    sgn, ctx = S
    _, h, eta, _ = I.testproblem_1d(n, 4.0, 1.0)
    hx = O.deriv(h, 1.0)
    Gd = O.dense_G_1d(eta, hx, 1.0)
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    for seed in range(3):
        u = np.random.default_rng(seed).standard_normal(n)
        Gu = torch.zeros(n, dtype=torch.float64, device="cuda")
        sgn.apply_operator(lay, dev(eta), dev(hx), dev(u), Gu)
        assert rel(host(Gu), Gd @ u) < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,eta0,hvar", [(96, 1.0, 1.0), (384, 4.0, 1.0), (1536, 1.0, 4.0),
                                         (6144, 1.0, 1.0), (30, 1.0, 1.0), (12288, 1.0, 1.0)])
def test_generic_pcg_testproblem(S, prec, n, eta0, hvar):
    """Eq:Testproblem (§6.2) at generic n: the CUDA solve equals the oracle's solution, and
    the float64 iteration count is the oracle's."""
    sgn, ctx = S
    _, h, eta, b = I.testproblem_1d(n, eta0, hvar)
    hx = O.deriv(h, 1.0)
    grid = O.make_grid(1, n, 1.0, 1.0)
    ref = O.solve_G(eta, hx, b, grid, rtol=1e-14, maxit=5000)[0]
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
    rtol = 1e-12 if prec == "fp64" else 1e-11
    info = sgn.pcg(lay, dev(eta), dev(hx), dev(b), x, rtol=rtol, maxit=5000, prec=p)[0]
    assert info["status"] == 0 and info["ratio"] <= rtol, info
    assert rel(host(x), ref) < (1e-10 if prec == "fp64" else 1e-9)
    if prec == "fp64":
        _, it12, _, _ = O.solve_G(eta, hx, b, grid, rtol=1e-12, maxit=5000)
        assert abs(info["iters"] - it12) <= 1
    else:
        assert info["refinements"] >= 1


def test_generic_pcg_ragged_batch_equals_alone(S):
    """A ragged batch of generic and power-of-two sizes: every instance reaches its known
    solution and equals the same instance solved alone, bitwise, in both precisions."""
    sgn, ctx = S
    cases = RAGGED[:8]
    F = [fields(n, L, 10 + i) for i, (n, L) in enumerate(cases)]
    hxs = [O.deriv(f[0], L) for f, (n, L) in zip(F, cases)]
    bs = [O.apply_G_1d(f[1], hx, f[2], L) for f, hx, (n, L) in zip(F, hxs, cases)]
    for prec in (sgn.PREC_FP64, sgn.PREC_MIXED):
        lay = sgn.Layout(ctx, [sgn.Grid(1, n, L) for n, L in cases])
        x = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(pack([f[1] for f in F])), dev(pack(hxs)), dev(pack(bs)), x,
                       rtol=1e-11, maxit=4000, prec=prec)
        xb = unpack(host(x), lay.offsets)
        for i, (n, L) in enumerate(cases):
            assert info[i]["status"] == 0, (n, info[i])
            assert rel(xb[i], F[i][2]) < 1e-8, n
            l1 = sgn.Layout(ctx, [sgn.Grid(1, n, L)])
            x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
            i1 = sgn.pcg(l1, dev(F[i][1]), dev(hxs[i]), dev(bs[i]), x1, rtol=1e-11, maxit=4000,
                         prec=prec)[0]
            assert np.array_equal(host(x1), xb[i]), n
            assert i1["iters"] == info[i]["iters"]


def test_generic_pcg_edge_cases(S):
    sgn, ctx = S
    n = 192
    _, h, eta, b = I.testproblem_1d(n, 1.0, 1.0)
    hx = O.deriv(h, 1.0)
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
    ref = np.linalg.solve(O.dense_G_1d(eta, hx, 1.0), b)
    for prec in (sgn.PREC_FP64, sgn.PREC_MIXED):
        x = dev(np.ones(n))
        info = sgn.pcg(lay, dev(eta), dev(hx), dev(np.zeros(n)), x, prec=prec)[0]
        assert info["status"] == 0 and info["iters"] == 0 and np.all(host(x) == 0.0)
        x = dev(ref)
        info = sgn.pcg(lay, dev(eta), dev(hx), dev(b), x, rtol=1e-9, prec=prec)[0]
        assert info["status"] == 0 and info["iters"] == 0
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(eta), dev(hx), dev(b), x, rtol=1e-14, maxit=2, prec=prec,
                       check=False)[0]
        assert info["status"] == 5 and info["iters"] <= 3
        bad = eta.copy()
        bad[7] = -0.2
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = sgn.pcg(lay, dev(bad), dev(hx), dev(b), x, prec=prec, check=False)[0]
        assert info["status"] == 7


def test_generic_gmres_matches_oracle(S):
    sgn, ctx = S
    cases = [(384, 1.0, 4.0, 1.0), (96, 1.0, 1.0, 1.0), (256, 1.0, 1.0, 1.0)]
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, L) for n, L, _, _ in cases])
    etas, hxs, bs, refs = [], [], [], []
    for n, L, eta0, hv in cases:
        _, h, eta, b = I.testproblem_1d(n, eta0, hv)
        hx = O.deriv(h, 1.0)
        etas.append(eta), hxs.append(hx), bs.append(b)
        refs.append(O.solve_G(eta, hx, b, O.make_grid(1, n, L, 1.0), rtol=1e-14, maxit=5000)[0])
    x = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
    info = sgn.gmres(lay, dev(pack(etas)), dev(pack(hxs)), dev(pack(bs)), x, rtol=1e-12,
                     restart=30, maxit=2000)
    for i, xi in enumerate(unpack(host(x), lay.offsets)):
        assert info[i]["status"] == 0 and info[i]["ratio"] <= 1e-12
        assert rel(xi, refs[i]) < 1e-10


def test_generic_rhs_matches_oracle(S):
    sgn, ctx = S
    cases = [(384, 200.0), (1536, 200.0), (96, 50.0), (6144, 400.0), (512, 100.0)]
    lay = sgn.Layout(ctx, [sgn.Grid(1, n, L, g=9.81) for n, L in cases])
    F = [fields(n, L, 30 + i) for i, (n, L) in enumerate(cases)]
    hxs = [O.deriv(f[0], L) for f, (n, L) in zip(F, cases)]
    fe = torch.zeros(lay.points, dtype=torch.float64, device="cuda")
    fU = torch.zeros_like(fe)
    sgn.rhs(lay, dev(pack([f[1] for f in F])), dev(pack([f[2] for f in F])),
            dev(pack([f[0] for f in F])), dev(pack(hxs)), fe, fU)
    fes, fUs = unpack(host(fe), lay.offsets), unpack(host(fU), lay.offsets)
    for i, (n, L) in enumerate(cases):
        h, eta, u = F[i]
        re, rU = O.rhs_1d(eta, u, h, hxs[i], L, 9.81)
        # third derivatives amplify float64 rounding: the bound is the oracle's own change
        # under a last-bit relative perturbation of its inputs
        rng = np.random.default_rng(i)
        jig = lambda a: a * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], a.size))
        pe, pU = O.rhs_1d(jig(eta), jig(u), h, jig(hxs[i]), L, 9.81)
        assert rel(fes[i], re) < max(1e-13, 20 * rel(pe, re)), n
        assert rel(fUs[i], rU) < max(1e-13, 20 * rel(pU, rU)), n


def _run(sgn, ctx, insts, scheme, nsteps, prec, rtol, order=4):
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g) for c in insts])
    eta = dev(pack([c.eta for c in insts]))
    u = dev(pack([c.u for c in insts]))
    h = dev(pack([c.h for c in insts]))
    U = torch.zeros_like(eta)
    gh = torch.zeros_like(eta)
    st = sgn.State(lay, eta, U, u, h, gh)
    st.init()
    p = sgn.PREC_FP64 if prec == "fp64" else sgn.PREC_MIXED
    dts = [c.dt for c in insts]
    if scheme == "rk4":
        st.rk4(dts, nsteps, rtol=rtol, prec=p)
    else:
        st.abk(order, dts, nsteps, rtol=rtol, prec=p)
    stats = st.stats()
    out = (unpack(host(eta), lay.offsets), unpack(host(U), lay.offsets),
           unpack(host(u), lay.offsets))
    st.close()
    return out, stats


def _oracle(c, scheme, nsteps, rtol, order=4):
    st = O.init_state(c.eta, c.u, c.h, O.make_grid(1, c.n, c.L, c.g))
    if scheme == "rk4":
        O.run_rk4(st, c.dt, nsteps, rtol)
    else:
        O.run_ab(st, order, c.dt, nsteps, rtol)
    return st


@pytest.mark.parametrize("scheme,order", [("rk4", 0), ("ab", 3)])
def test_generic_steppers_shelf_fp64_match_oracle(S, scheme, order):
    sgn, ctx = S
    c = I.shelf_case(n=384, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0, dt=0.02)
    (eta, U, u), stats = _run(sgn, ctx, [c], scheme, 20, "fp64", 1e-13, order or 4)
    ref = _oracle(c, scheme, 20, 1e-13, order or 4)
    assert rel(eta[0] - c.h, ref.eta - c.h) < 1e-10
    assert rel(u[0], ref.u) < 1e-10 and rel(U[0], ref.U) < 1e-10
    assert stats["status"] == 0


def test_generic_rk4_solitary_wave_and_mixed_precision(S):
    """A solitary wave on n = 1536 (flat bottom): float64 RK4 against the oracle and the
    closed form; mixed RK4 within 1e-6 of float64; in a batch with a power of two the
    generic instance steps exactly as alone."""
    sgn, ctx = S
    c = I.solitary_case(n=1536, L=150.0, a=0.2, x0=40.0, dt=0.02)
    (eta, U, u), stats = _run(sgn, ctx, [c], "rk4", 20, "fp64", 1e-12)
    ref = _oracle(c, "rk4", 20, 1e-13)
    assert rel(eta[0], ref.eta) < 1e-11 and rel(u[0], ref.u) < 1e-10
    x = I.grid_1d(c.n, c.L)
    ee, _ = I.solitary_wave_1d(x, c.L, 1.0, 0.2, 40.0, c.g, t=20 * 0.02)
    assert np.abs(eta[0] - ee).max() < 1e-6
    assert stats["status"] == 0 and stats["solves"] == 20 * 4
    (em, _, um), sm = _run(sgn, ctx, [c], "rk4", 20, "mixed", 1e-11)
    assert rel(em[0], ref.eta) < 1e-6 and rel(um[0], ref.u) < 1e-6 and sm["status"] == 0
    d = I.shelf_case(n=512, L=200.0, a=0.3, x0=40.0, r=0.5, xs=45.0, dt=0.02)
    (eb, _, ub), _ = _run(sgn, ctx, [d, c], "rk4", 3, "mixed", 1e-10)
    (e1, _, u1), _ = _run(sgn, ctx, [c], "rk4", 3, "mixed", 1e-10)
    assert np.array_equal(eb[1], e1[0]) and np.array_equal(ub[1], u1[0])


def test_generic_size_rejections(S):
    sgn, ctx = S
    for n in (7, 14, 98, 4, 15, 18432, 32768):
        with pytest.raises(sgn.SgnError) as e:
            sgn.Layout(ctx, [sgn.Grid(1, n, 1.0)])
        assert e.value.status == 2, n
    c = I.shelf_case(n=96, L=50.0, a=0.2, x0=10.0, r=0.5, xs=25.0, dt=0.02)
    lay = sgn.Layout(ctx, [sgn.Grid(1, c.n, c.L, g=c.g)])
    eta, u, h = dev(c.eta), dev(c.u), dev(c.h)
    st = sgn.State(lay, eta, torch.zeros_like(eta), u, h, torch.zeros_like(eta))
    st.init()
    with pytest.raises(sgn.SgnError):
        st.set_dealias(True)
    with pytest.raises(sgn.SgnError):
        st.linimp([c.dt], 1)
    with pytest.raises(sgn.SgnError):
        st.rk4_nc([c.dt], 1)
    st.close()
